"""The C ABI library builds, loads on the CPU host and exports every function the header
declares (no compute calls: there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wsbm_hss.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wsbm_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_api():
    names = declared_functions()
    for must in ("wsbm_create", "wsbm_factor", "wsbm_solve", "wsbm_farfield", "wsbm_entries",
                 "wsbm_entries_raw", "wsbm_hankel01", "wsbm_proxy_block", "wsbm_rhs_planewave",
                 "wsbm_stats", "wsbm_destroy", "wsbm_strerror", "wsbm_box_info"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2607_00790_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    lib = ctypes.CDLL(build.LIB)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    lib.wsbm_strerror.restype = ctypes.c_char_p
    assert lib.wsbm_strerror(-4) == b"interpolative decomposition rank above its cap"


def test_set_allocator_arguments():
    """wsbm_set_allocator touches no device: both callbacks or neither."""
    from paper_2607_00790_gb300 import binding
    L = binding.lib()
    none_a, none_f = binding._ALLOC_FN(), binding._FREE_FN()
    one = binding._ALLOC_FN(lambda n, s, c: None)
    assert L.wsbm_set_allocator(one, none_f, None) == -1  # WSBM_ERR_INVALID_ARG
    binding.use_torch_allocator(True)
    binding.use_torch_allocator(False)
    assert L.wsbm_set_allocator(none_a, none_f, None) == 0


LAYOUT_C = r"""
#include <stddef.h>
#include <stdio.h>
#include "wsbm_hss.h"
#define F(T, m) printf("%s.%s %zu\n", #T, #m, offsetof(T, m));
int main(void) {
  printf("wsbm_geom %zu\nwsbm_params %zu\nwsbm_stats_t %zu\n", sizeof(wsbm_geom),
         sizeof(wsbm_params), sizeof(wsbm_stats_t));
  F(wsbm_params, id_tol) F(wsbm_params, precision) F(wsbm_params, proxy_ratio)
  F(wsbm_params, max_levels) F(wsbm_params, root_cap) F(wsbm_params, id_method)
  F(wsbm_params, formulation)
  F(wsbm_stats_t, ms_entries) F(wsbm_stats_t, max_rank) F(wsbm_stats_t, rank_per_level)
  F(wsbm_stats_t, factor_bytes) F(wsbm_stats_t, ms_proxy) F(wsbm_stats_t, launches)
  return 0;
}
"""


def test_struct_layout_matches_binding(tmp_path):
    import subprocess
    from paper_2607_00790_gb300 import binding
    src = tmp_path / "layout.c"
    src.write_text(LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    assert int(got["wsbm_geom"]) == ctypes.sizeof(binding.Geom)
    assert int(got["wsbm_params"]) == ctypes.sizeof(binding.Params)
    assert int(got["wsbm_stats_t"]) == ctypes.sizeof(binding.Stats)
    for key, val in got.items():
        if "." in key:
            T, m = key.split(".")
            cls = {"wsbm_params": binding.Params, "wsbm_stats_t": binding.Stats}[T]
            assert getattr(cls, m).offset == int(val), key
