// kernels.cuh -- internal interfaces between the library's translation units.
#pragma once

#include <vector>

#include "common.cuh"

namespace obk {

// Stage clock of obk_create: CUDA events recorded on the setup stream.
struct StageClock {
    static constexpr int kMax = 16;
    cudaEvent_t ev[kMax] = {};
    int n = 0;
    cudaStream_t st = nullptr;
    void mark(cudaStream_t s)
    {
        if (n >= kMax) return;
        st = s;
        if (!ev[n]) cudaEventCreate(&ev[n]);
        cudaEventRecord(ev[n], s);
        ++n;
    }
    // milliseconds between consecutive marks (n - 1 values)
    int read(double* ms, int cap)
    {
        if (n < 2) return 0;
        cudaEventSynchronize(ev[n - 1]);
        int k = 0;
        for (int i = 1; i < n && k < cap; ++i, ++k) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[i - 1], ev[i]);
            ms[k] = t;
        }
        return k;
    }
    ~StageClock()
    {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    }
};

struct RcmStats {
    int64_t components = 0;
    int64_t levels = 0;
    int64_t gl_rounds = 0;
    int64_t graph_edges = 0;
};

// perm[k] = vertex placed at position k by Reverse Cuthill-McKee (rcm.cu).
// With a clock, marks the end of: the symmetric graph, the rank orders, the
// pseudo-peripheral search and the Cuthill-McKee order.
void rcm_reorder(int64_t N, const int64_t* rp, const int32_t* ci, int64_t nnz, int32_t* perm,
                 long long spin_limit, int* d_err, RcmStats* stats, cudaStream_t st,
                 StageClock* clock = nullptr);

// Sorted neighbour lists of pattern(A + A^T) without self loops (rcm.cu).
void build_sym_graph(int64_t N, const int64_t* rp, const int32_t* ci, int64_t nnz, DBuf<int64_t>& gp,
                     DBuf<int32_t>& adj, cudaStream_t st);

// ---- setup.cu ---------------------------------------------------------------

// Returns nonzero flags in *d_bad if the CSR is malformed (see obk.h).
void validate_csr(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                  int64_t nnz, int* d_bad, cudaStream_t st);

int64_t half_bandwidth(int64_t N, const int64_t* rp, const int32_t* ci, int64_t nnz, cudaStream_t st);

// Longest segment max_i (ptr[i+1] - ptr[i]) of a pointer array of n segments.
int64_t max_segment_length(int64_t n, const int64_t* ptr, cudaStream_t st);

// A~ = P A P^T with sorted columns.
void permute_csr(int64_t N, const int64_t* rp, const int32_t* ci, const double* v, int64_t nnz,
                 const int32_t* perm, int32_t* iperm, int64_t* rp_t, int32_t* ci_t, double* v_t,
                 cudaStream_t st);

// Everything the sweep needs, in device memory.
// Mirror slices of a (group, tile) piece with at least kMirrorDoubleMin
// column segments hold two segments per lane, entries interleaved (the
// sweep's phase 2 folds both of a lane's columns in one pass over its
// entries); a smaller piece keeps one segment per lane, so that its few
// slices still spread over a block's warps.
constexpr int64_t kMirrorDoubleMin = 4096;
constexpr int32_t kOneColumn = -2;  // second column word of a one-column mirror slice

struct SweepLayout {
    int64_t N = 0, nnz = 0;
    int64_t G = 0;          // groups
    int64_t Ngm = 0;        // rows that belong to a group (nonzero rows)
    int64_t nseg = 0;       // (group, column) segments of the column mirror
    int64_t nnz_gm = 0;     // entries of grouped rows
    int64_t n_conflicts = 0;
    int64_t color_rounds = 0;  // rounds of the fixed-point colouring
    // group-major CSR: rows of group 0, then group 1, ...  The row pointers
    // are always built; the entries (grp_ci, grp_v, grp_v32) only on first use
    // by ensure_gm_csr (the sub-warp sweeps, the batch kernel, the Gram entries
    // and the cosine statistics read them; the sliced sweep does not), copied
    // from the permuted matrix src_* that the handle keeps.
    DBuf<int64_t> grp_rp;   // Ngm+1
    DBuf<int32_t> grp_ci;   // nnz_gm (columns in permuted numbering)
    DBuf<double> grp_v;     // nnz_gm
    DBuf<float> grp_v32;    // nnz_gm (precision form)
    bool has_gm_csr = false;
    bool want_fp32 = false;
    const int64_t* src_rp = nullptr;  // the permuted matrix A~ (owned by the handle)
    const int32_t* src_ci = nullptr;
    const double* src_v = nullptr;
    DBuf<double> grp_inv;   // Ngm, 1 / ||A_i||^2
    DBuf<float> grp_inv32;  // Ngm
    DBuf<int32_t> grp_row;  // Ngm, permuted row index of each group-major row
    DBuf<int64_t> gptr;     // G+1 (device)
    std::vector<int64_t> h_gptr;
    // column mirror for the x update: entries ordered by (group, column, row);
    // seg_order lists the segments in the order of the sliced copy (group,
    // tile of the column, length, column)
    DBuf<int64_t> gseg_ptr; // G+1, first segment of each group
    std::vector<int64_t> h_gseg_ptr;
    DBuf<int64_t> seg_ptr;  // nseg+1, first mirror entry of each segment
    DBuf<int32_t> seg_col;  // nseg
    DBuf<int32_t> mir_row;  // nnz_gm, group-major row index
    DBuf<double> mir_val;   // nnz_gm
    DBuf<float> mir_val32;  // nnz_gm
    DBuf<uint32_t> seg_order;  // nseg
    // Sliced ELL (SELL-32) copies for the persistent sweep.  Inside each group
    // the rows (and the mirror segments) are cut into slices of 32 in their
    // (length, index) order; a slice stores entry j of its 32 rows next to each
    // other (position base + 32 j + lane), rows shorter than the slice's
    // longest padded with value 0 and index 0.
    int64_t ns = 0, nms = 0;         // row slices, mirror slices
    int64_t sell_nnz = 0, msell_nnz = 0;
    std::vector<int64_t> h_sl_gptr;  // G+1, first row slice of each group
    std::vector<int64_t> h_ml_gptr;  // G+1, first mirror slice of each group
    DBuf<int64_t> sl_gptr, ml_gptr;  // device copies of the two
    // off-diagonal Gram entries of each group (rows of one group sharing a
    // column), partners ascending; built on the first solve with pinv_iters > 0
    bool has_gram = false;
    DBuf<int64_t> gram_ptr;          // Ngm+1
    DBuf<int32_t> gram_idx;          // group-major partner index
    DBuf<double> gram_val;           // A_i . A_j
    DBuf<int64_t> sl_ptr;            // ns+1, first entry of each row slice
    DBuf<int64_t> sl_row0;           // ns, group-major index of the slice's first row
    DBuf<int32_t> sl_nrow;           // ns, rows in the slice (32 except a group's last)
    DBuf<int32_t> sci;               // sell_nnz, column indices
    DBuf<double> sv;                 // sell_nnz
    DBuf<float> sv32;                // sell_nnz (precision form)
    DBuf<int64_t> ml_ptr;            // nms+1
    DBuf<int32_t> mcol;              // 64 nms: the two columns of each slice lane (-1: none)
    DBuf<int32_t> mrow;              // msell_nnz, group-major row index
    DBuf<double> mv;                 // msell_nnz
    DBuf<float> mv32;                // msell_nnz
    // Tiles: T ranges of B consecutive permuted rows (and columns).  The layout
    // is ordered by (group, tile) first: rows of group g in tile t are the
    // group-major rows [gt_ptr[g*T + t], gt_ptr[g*T + t + 1]) and their slices
    // [sl_tptr[g*T + t], sl_tptr[g*T + t + 1]); the mirror segments of the
    // columns of tile t likewise (gts_ptr, ml_tptr).  reach_lo/hi[t] = the
    // lowest/highest tile with a column of a row of tile t or a row of a column
    // of tile t (t itself included): the tiles whose work a step of tile t
    // depends on.
    int64_t T = 1, B = 1;
    DBuf<int64_t> gt_ptr, gts_ptr;          // G*T + 1 (device)
    std::vector<int64_t> h_sl_tptr, h_ml_tptr;  // G*T + 1
    DBuf<int64_t> sl_tptr, ml_tptr;         // device copies
    std::vector<int32_t> h_ml_pdbl;             // G*T: the piece's mirror slices hold two segments per lane
    DBuf<int32_t> reach_lo, reach_hi;       // T
    // largest staging windows of a one-tile block: x columns of its reach, and
    // group-major rows of one group in its reach
    int64_t xwin_max = 0, ywin_max = 0;
    // permuted-order results kept for inspection
    DBuf<double> nsq;       // N
    DBuf<int32_t> group_of; // N
};

// Row norms, pair cosines, greedy first-fit groups and the sweep layout
// (paper Section 3.3 at one row per block).
void group_build(int64_t N, const int64_t* rp, const int32_t* ci, const double* v, int64_t nnz,
                 double thr, long long spin_limit, int* d_err, SweepLayout& L, bool want_fp32,
                 cudaStream_t st, StageClock* clock = nullptr);

// Column lists of a CSR matrix (nrows x ncols, columns sorted in each row):
// cptr[ncols+1], rows ascending inside each column with their values, and the
// column-list position of every CSR entry (setup.cu).
void build_csc(int64_t nrows, int64_t ncols, const int64_t* rp, const int32_t* ci, const double* v, int64_t nnz,
               DBuf<int64_t>& cptr, DBuf<int32_t>& crow, DBuf<double>& cval, DBuf<int64_t>& pos_of,
               cudaStream_t st);

// ---- blocks.cu: the paper-literal block form (Section 3.3, Algorithm 4) ----------

struct BlockArgs {
    int k = 8;
    double thr = 0.1;
    int inner_max = 500;
    double inner_tol = 1e-13;
    double tol = 1e-8;
    int64_t maxit = 1000;
    long long spin_limit = 0;
};
struct BlockResult {
    int64_t iters = 0;
    int64_t cgls_steps = 0;
    double rel_res = 0.0;
    int status = 1;
    int n_pairs = 0, n_nclass = 0;
};
// On A~ (N x N CSR, RCM order) with its column lists, f~ and x~ (updated in place).
BlockResult run_blocks(int64_t N, const int64_t* rp, const int32_t* ci, const double* v, const int64_t* cptr,
                       const int32_t* crow, const double* cval, const double* ft, double* xt, const BlockArgs& a,
                       int* d_err, cudaStream_t st);

// Builds the entries of the group-major CSR if not yet built (setup.cu).
void ensure_gm_csr(SweepLayout& L, cudaStream_t st);

// Off-diagonal Gram entries of every group of a built layout (setup.cu).
void build_group_gram(SweepLayout& L, int* d_err, cudaStream_t st);

// Row cosine-table statistics of a built layout (Definitions 1-2 at the row
// level): nonzero entries and the sum of |cos| in units of 2^-32 (setup.cu).
void cosine_stats(SweepLayout& L, int64_t* nz, uint64_t* sum, int* d_err, cudaStream_t st);

// ---- sweep.cu -----------------------------------------------------------------

struct SolveArgs {
    int precision = 0;
    int check_every = 1;  // < 0: adaptive schedule
    int pinv_iters = 0;   // > 0: Jacobi steps of the Eq. 1.3 group projection (FP64)
    int inner_sweeps = 0;
    int max_outer = 100;
    double stagnation = 0.0;
    double tol = 1e-8;
    int64_t maxit = 1000;
    long long spin_limit = kDefaultSpins;
    int sub = 0;  // lanes per row (0 = choose)
    int sync_mode = 1;  // 1 = grid barriers between the phases, 2 = band-local step counters
    int staging = 0;    // band-local sweep: 1 = x and y windows in shared memory when worth it, 0 or 2 = never
    int block = 1024;   // threads per block of the sweep kernel: 1024 (one per SM) or 512 (two per SM)
};

struct SolveResult {
    int status = 0;
    int64_t sweeps = 0;
    int64_t outer = 0;
    double rel_res = 0.0;
    double sweep_ms = 0.0;
};

// Device time (ms) of one sweep with `sub` lanes per row (0 = default rule),
// `block` threads per block and the given staging mode, measured on zero
// vectors as the difference of 2- and 8-sweep solves.
double time_sweep(const SweepLayout& L, int sub, int precision, int block, int staging, int sync_mode, int* d_err,
                  cudaStream_t st);

// A setting of the sweep kernel chosen by the autotuner (sub = 0: none).
struct TuneChoice {
    int sub = 0;      // lanes per row
    int block = 0;    // threads per block
    int staging = 0;  // 1 = staged windows in shared memory, 2 = global memory
    int sync = 0;     // 1 = grid barriers, 2 = band-local step counters
};

// Ordering used when neither the options nor the autotuner fix it: band-local
// counters only for systems whose layout fills every tile of the GPU and that
// have few groups (each counter step costs more than a barrier on a small grid).
int default_sync_mode(const SweepLayout& L);

// Lanes per row chosen by the fixed rule from the mean row length.
int choose_sub(double avg_row);

// Number of tiles of the sweep layout of an N-row system on the current device:
// two per SM (a block of the persistent sweep owns one or two), fewer for
// small systems (one per 2048 rows).
int64_t sweep_tiles(int64_t N);

// x (N, permuted order) is updated in place; f_gm (Ngm) is f in group-major
// order; fnorm2 = ||f~||^2 and zero_f2 = sum of f_i^2 over all-zero rows.
SolveResult run_solve(const SweepLayout& L, const double* f_gm, double fnorm2, double zero_f2,
                      double* x, const SolveArgs& a, int* d_err, cudaStream_t st);

}  // namespace obk
