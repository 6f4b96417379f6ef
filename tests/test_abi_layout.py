"""The ctypes structures of the Python binding have the sizes and field offsets
of the C structures in include/obk.h (a small C program compiled with gcc
against the header prints them).  CPU only."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C struct name -> (binding attribute, fields)
STRUCTS = {
    "obk_csr": ("_Csr", ["row_ptr", "col_idx", "val", "nnz", "device_ptrs"]),
    "obk_opts": ("Opts", ["precision", "check_every", "inner_sweeps", "max_outer", "stagnation",
                          "timeout_spins", "rows_per_warp", "pinv_iters", "sync_mode", "staging", "block_threads",
                          "reserved"]),
    "obk_info": ("_Info", ["sweeps", "rel_res", "setup_ms", "solve_ms", "groups", "bandwidth_before",
                           "bandwidth_after", "outer_iters", "sweep_ms", "n_conflicts", "status"]),
    "obk_block_opts": ("BlockOpts", ["k", "inner_max", "thr", "inner_tol", "n_pairs", "n_nclass", "cgls_steps"]),
    "obk_gstats": ("_GStats", ["N", "nonzero_entries", "abs_cos_sum", "zn", "nn", "groups", "min_group_rows",
                               "max_group_rows", "conflicts", "color_rounds"]),
    "obk_tune": ("_Tune", ["rows_per_warp", "block_threads", "staging", "sync_mode", "n_candidates",
                           "sweep_ms", "candidate_ms"]),
    "obk_thr_probe": ("_ThrProbe", ["thr", "groups", "conflicts", "probe_sweeps", "setup_ms", "probe_ms", "rel_res",
                                     "rate", "predicted_ms"]),
    "obk_peaks": ("_Peaks", ["fp64_fma_tflops", "fp32_fma_tflops", "l2_gather_g_per_s", "l2_read_gbs",
                             "int64_mad_tops", "int32_mad_tops"]),
}


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "obk.h"', "int main(void) {"]
    for s, (_, fields) in STRUCTS.items():
        lines.append(f'    printf("{s} sizeof %zu\\n", sizeof({s}));')
        for f in fields:
            lines.append(f'    printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        s, f, v = line.split()
        layout[(s, f)] = int(v)
    return layout


def test_binding_structs_match_header(tmp_path):
    import paper_2401_00672_gb300 as obk  # noqa: F401  (needs the built library)

    layout = _c_layout(tmp_path)
    for s, (attr, fields) in STRUCTS.items():
        cls = getattr(obk, attr)
        assert ctypes.sizeof(cls) == layout[(s, "sizeof")], s
        for f in fields:
            assert getattr(cls, f).offset == layout[(s, f)], (s, f)
