"""Host checks of two algorithmic facts the GPU setup relies on (CPU only):

* first fit in index order is the unique fixed point of
  c_i = mex{c_j : j < i conflicting}, reached by in-place rounds in any row
  order and with any run structure (the grouping kernel's rounds);
* the odd-even merge sorting networks of the per-segment sort (the product
  source, compiled for the host) sort every input (0-1 principle for 8 and 16
  inputs, random inputs for 32 and 64).
"""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _first_fit(n, earlier):
    c = np.zeros(n, np.int64)
    for i in range(n):
        used = {c[j] for j in earlier[i]}
        g = 0
        while g in used:
            g += 1
        c[i] = g
    return c


def _rounds(n, earlier, order_rng, run):
    c = np.zeros(n, np.int64)
    rounds = 0
    while True:
        rounds += 1
        changed = False
        starts = np.arange(0, n, run)
        order_rng.shuffle(starts)  # lane groups finish their runs in any order
        for s in starts:
            for i in range(s, min(s + run, n)):  # a run in index order
                used = {c[j] for j in earlier[i]}
                g = 0
                while g in used:
                    g += 1
                if g != c[i]:
                    c[i] = g
                    changed = True
        if not changed:
            return c, rounds
        assert rounds <= n + 2


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("run", [1, 3, 8])
def test_fixed_point_rounds_reach_first_fit(seed, run):
    rng = np.random.default_rng(seed)
    n = 120
    # conflicts mostly between nearby rows, a few long-range ones
    earlier = [[] for _ in range(n)]
    for i in range(n):
        for j in range(max(0, i - 6), i):
            if rng.random() < 0.4:
                earlier[i].append(j)
        if i > 20 and rng.random() < 0.2:
            earlier[i].append(int(rng.integers(0, i - 10)))
    want = _first_fit(n, earlier)
    got, _ = _rounds(n, earlier, np.random.default_rng(seed + 100), run)
    assert np.array_equal(got, want)


def _network_source():
    src = open(os.path.join(ROOT, "paper_2401_00672_gb300", "csrc", "primitives.cu")).read()
    a = src.index("__device__ __forceinline__ void cmp_swap(")
    b = src.index("template <int W>\n__device__ __forceinline__ void sort_segment(")
    return re.sub(r"#pragma unroll\n", "", src[a:b])


def test_sorting_networks(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    prog = (
        "#include <cstdint>\n#include <cstdio>\n#include <algorithm>\n#include <random>\n"
        "#define __device__\n#define __forceinline__ inline\n"
        + _network_source()
        + r"""
template <int W> bool zero_one() {
  for (uint32_t m = 0; m < (1u << W); ++m) {
    uint64_t a[W]; for (int t = 0; t < W; ++t) a[t] = (m >> t) & 1;
    oddeven_sort<W>(a);
    for (int t = 1; t < W; ++t) if (a[t - 1] > a[t]) return false;
  }
  return true;
}
template <int W> bool random_inputs() {
  std::mt19937_64 g(7);
  for (int r = 0; r < 20000; ++r) {
    uint64_t a[W], b[W];
    for (int t = 0; t < W; ++t) a[t] = b[t] = g() % 97;
    oddeven_sort<W>(a); std::sort(b, b + W);
    for (int t = 0; t < W; ++t) if (a[t] != b[t]) return false;
  }
  return true;
}
int main() {
  bool ok = zero_one<8>() && zero_one<16>() && random_inputs<32>() && random_inputs<64>();
  std::printf("%s\n", ok ? "ok" : "fail");
  return ok ? 0 : 1;
}
""")
    cpp = tmp_path / "net.cpp"
    cpp.write_text(prog)
    exe = tmp_path / "net"
    subprocess.run([cxx, "-O1", "-std=c++17", str(cpp), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok"


def _conflict_source():
    src = open(os.path.join(ROOT, "paper_2401_00672_gb300", "csrc", "setup.cu")).read()
    a = src.index("__device__ __forceinline__ bool is_conflict(")
    b = src.index("// x == 0.0 for a row norm")
    return src[a:b]


def test_conflict_band_matches_ieee_division(tmp_path):
    """The integer band test of the pair kernel decides |dot / (s_j s_i)| >= thr
    exactly like the IEEE division, also for dot products within a few units of
    rounding of the threshold."""
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    prog = (
        "#include <cstdint>\n#include <cstdio>\n#include <cstring>\n#include <cmath>\n#include <random>\n"
        "#define __device__\n#define __forceinline__ inline\n"
        "static inline long long __double_as_longlong(double x) { long long r; std::memcpy(&r, &x, 8); return r; }\n"
        "static inline double __ddiv_rn(double a, double b) { return a / b; }\n"
        "static inline double __dmul_rn(double a, double b) { return a * b; }\n"
        + _conflict_source()
        + r"""
int main() {
  std::mt19937_64 g(11);
  std::uniform_real_distribution<double> u(-3.0, 3.0), w(0.0, 1.0);
  long long n = 0, bad = 0;
  const double thrs[4] = {0.1, 0.05, 0.3, 0.7};
  for (int r = 0; r < 200000; ++r) {
    double si = std::pow(10.0, u(g)), sj = std::pow(10.0, u(g));
    double thr = r % 5 == 4 ? w(g) * 0.9 + 0.01 : thrs[r % 4];
    double thr_si = thr * si;
    double t = thr_si * sj;
    for (int k = -40; k <= 40; ++k) {
      double dot = std::nextafter(t, k < 0 ? 0.0 : INFINITY);
      for (int s = 1; s < (k < 0 ? -k : k); ++s) dot = std::nextafter(dot, k < 0 ? 0.0 : INFINITY);
      if (k == 0) dot = t;
      for (int sign = 0; sign < 2; ++sign) {
        double d = sign ? -dot : dot;
        bool want = std::fabs(d / (sj * si)) >= thr;
        if (is_conflict(d, sj, si, thr_si, thr) != want) ++bad;
        ++n;
      }
    }
    double d = (w(g) - 0.5) * 4.0 * t;
    if (is_conflict(d, sj, si, thr_si, thr) != (std::fabs(d / (sj * si)) >= thr)) ++bad;
    ++n;
  }
  std::printf("%lld %lld\n", n, bad);
  return bad == 0 ? 0 : 1;
}
""")
    cpp = tmp_path / "band.cpp"
    cpp.write_text(prog)
    exe = tmp_path / "band"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", str(cpp), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    n, bad = map(int, r.stdout.split())
    assert n > 1_000_000 and bad == 0, r.stdout


def _cm_sequential(adj, rank, root):
    order, seen = [root], {root}
    k = 0
    while k < len(order):
        u = order[k]
        for w in sorted(adj[u], key=lambda v: rank[v]):
            if w not in seen:
                seen.add(w)
                order.append(w)
        k += 1
    return order


def _cm_by_claims(adj, rank, root):
    # the GPU formulation: every placed vertex has priority P (the root 0; the
    # idx-th child, in rank order, of the vertex at queue position k gets
    # (k + 1) * 2^32 + idx); each vertex of the next level is claimed by the
    # smallest priority among its placed neighbours; a level's children are
    # counted per parent and placed after a scan of the counts
    INF = float("inf")
    claim = {v: INF for v in adj}
    prio = {root: 0}
    Q = [root]
    claim[root] = 0
    for x in adj[root]:
        claim[x] = min(claim[x], 0)
    lo, hi = 0, 1
    while hi > lo:
        counts = []
        kids = []
        for k in range(lo, hi):
            u = Q[k]
            ch = [w for w in sorted(adj[u], key=lambda v: rank[v]) if claim[w] == prio[u] and w not in prio]
            counts.append(len(ch))
            kids.append(ch)
        for k, ch in zip(range(lo, hi), kids):
            for idx, w in enumerate(ch):
                prio[w] = (k + 1) * 2**32 + idx
                Q.append(w)
        for w in Q[hi:]:
            for x in adj[w]:
                claim[x] = min(claim[x], prio[w])
        lo, hi = hi, len(Q)
    return Q


@pytest.mark.parametrize("seed", range(8))
def test_cuthill_mckee_by_claims_equals_sequential(seed):
    rng = np.random.default_rng(seed)
    n = 200
    adj = {v: set() for v in range(n)}
    for v in range(1, n):  # a random tree keeps the graph connected
        u = int(rng.integers(0, v))
        adj[u].add(v)
        adj[v].add(u)
    for _ in range(3 * n):
        a, b = map(int, rng.integers(0, n, 2))
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    rank = {v: r for r, v in enumerate(sorted(adj, key=lambda v: (len(adj[v]), v)))}
    root = int(rng.integers(0, n))
    assert _cm_by_claims(adj, rank, root) == _cm_sequential(adj, rank, root)
