// batch.cuh -- one thread block per system (batch.cu).
#pragma once

#include <stdint.h>

#include "common.cuh"

struct obk_handle;

namespace obk {

// Whether obk_solve_batch can take this system (capi.cu).
bool batch_eligible(const obk_handle* h);

// Builds what the batch kernel reads (the group-major rows) on the handle's
// own stream, without waiting (capi.cu); obk_solve_batch does it otherwise.
void prepare_batch(obk_handle* h);

// The stream a handle was created on (capi.cu).
void* handle_stream(const obk_handle* h);

// Everything one block needs to solve one prepared system (device pointers).
struct BatchSystem {
    int64_t m, n, N, Ngm, G, n_zero;
    const int32_t* perm;      // N
    const int32_t* src_gm;    // Ngm
    const int32_t* zero_src;  // n_zero
    const int64_t* gptr;      // G+1
    const int64_t* gseg_ptr;  // G+1
    const int64_t* grp_rp;
    const int32_t* grp_ci;
    const double* grp_v;
    const double* grp_inv;
    const int64_t* seg_ptr;
    const int32_t* seg_col;
    const int32_t* mir_row;
    const double* mir_val;
    const double* f;          // m
    const double* x0;         // n or nullptr
    double* x_out;            // n
    double tol, stagnation;
    int64_t maxit;
    int64_t check_every;      // > 0 fixed cadence, < 0 adaptive
    double* result;           // [0] status (0 ok, 1 not converged), [1] sweeps, [2] rel. residual
};

// Shared memory one system needs (x, y and f in group-major order).
size_t batch_smem_bytes(int64_t N, int64_t Ngm);
size_t batch_smem_limit();
void launch_batch(const BatchSystem* d_systems, int count, size_t smem, cudaStream_t st);

}  // namespace obk
