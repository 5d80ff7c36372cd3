"""CPU checks of the C ABI: the library builds and loads, exports every entry
point the public headers declare, the ctypes mirrors of the structs match the
C layout, and error paths return statuses (no GPU is touched)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("pdd.h", "pdd_debug.h")]


@pytest.fixture(scope="module")
def libpdd():
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    return pdd


def _declared(header):
    src = open(header).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pdd_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(libpdd):
    lib = libpdd.lib()
    names = [n for h in HEADERS for n in _declared(h)]
    assert "pdd_estimate_nodes" in names and "pdd_set_control_grid" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared but not exported"
    bound = {s[0] for s in libpdd._SIGS}
    assert set(names) <= bound, f"binding lacks {set(names) - bound}"


def test_struct_layouts_match_header(libpdd, tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "pdd.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(pdd_problem_desc), sizeof(pdd_grid_desc),
         sizeof(pdd_estimate_args), sizeof(pdd_node_stats));
  printf("%zu %zu %zu %zu %zu %zu\\n", offsetof(pdd_estimate_args, n_paths),
         offsetof(pdd_estimate_args, seed), offsetof(pdd_estimate_args, flags),
         offsetof(pdd_estimate_args, path_steps), offsetof(pdd_node_stats, mean_steps),
         offsetof(pdd_node_stats, n_truncated));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split()
    got = list(map(int, out))
    P = libpdd
    want = [ctypes.sizeof(P.ProblemDesc), ctypes.sizeof(P.GridDesc),
            ctypes.sizeof(P.EstimateArgs), ctypes.sizeof(P.NodeStats),
            P.EstimateArgs.n_paths.offset, P.EstimateArgs.seed.offset,
            P.EstimateArgs.flags.offset, P.EstimateArgs.path_steps.offset,
            P.NodeStats.mean_steps.offset, P.NodeStats.n_truncated.offset]
    assert got == want


def test_error_paths_without_gpu(libpdd):
    lib = libpdd.lib()
    assert lib.pdd_abi_version() == 1
    assert lib.pdd_estimate_nodes(None, None, None) == libpdd.PDD_ERR_INVALID
    assert b"NULL" in lib.pdd_last_error()
    assert lib.pdd_create_problem(None, None, None) == libpdd.PDD_ERR_INVALID
    assert lib.pdd_ctx_set_timing(None, 1) == libpdd.PDD_ERR_INVALID
    assert lib.pdd_ctx_abort(None) == libpdd.PDD_ERR_INVALID
    assert lib.pdd_debug_philox(None, None, None, -1) == libpdd.PDD_ERR_INVALID
    lib.pdd_ctx_destroy(None)  # no-op
    assert lib.pdd_destroy_problem(None) == libpdd.PDD_OK
    h = ctypes.c_void_p()
    st = lib.pdd_ctx_create(0, None, 0, ctypes.byref(h))
    import torch
    if not torch.cuda.is_available():
        assert st < 0 and h.value is None
        assert len(lib.pdd_last_error()) > 0
    else:
        assert st == 0
        lib.pdd_ctx_destroy(h)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1512_02818_gb300 import pdd
    monkeypatch.setattr(pdd, "_lib", None)
    monkeypatch.setattr(pdd, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        pdd.lib()
