"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every function that include/proxsdp_gpu.h declares, and the ctypes structs
match the C layout.  No compute calls (there is no GPU here)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "proxsdp_gpu.h")


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_05231_gb300 as pkg

    return pkg


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(proxsdp_gpu_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["proxsdp_gpu_create", "proxsdp_gpu_set_problem", "proxsdp_gpu_solve",
                 "proxsdp_gpu_get_primal_dual", "proxsdp_gpu_destroy", "proxsdp_gpu_last_error"]:
        assert want in names


def test_library_exports_every_declared_symbol(built):
    L = built.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", built._binding.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (proxsdp_gpu_\w+)", out))
    assert set(declared_functions()) <= exported
    assert set(built.EXPORTED) == set(declared_functions())


def test_struct_layout_matches_c(built):
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "proxsdp_gpu.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(proxsdp_gpu_settings), offsetof(proxsdp_gpu_settings, lanczos_tol),
         offsetof(proxsdp_gpu_settings, use_graphs), sizeof(proxsdp_gpu_info), offsetof(proxsdp_gpu_info, norm_M),
         offsetof(proxsdp_gpu_settings, memory_limit_bytes), offsetof(proxsdp_gpu_settings, at_max_rank));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    S, I = built.Settings, built.Info
    assert vals == [ctypes.sizeof(S), S.lanczos_tol.offset, S.use_graphs.offset, ctypes.sizeof(I), I.norm_M.offset,
                    S.memory_limit_bytes.offset, S.at_max_rank.offset]


def test_settings_defaults_without_gpu(built):
    s = built.default_settings()
    assert s.tol == 1e-4 and s.rank_init == 8 and s.block_size == 16 and s.window == 100
    assert abs(s.alpha_frac - 0.95) < 1e-15 and s.normalize_rows == 1
    assert s.max_rank == 64 and s.at_max_rank == 0 and s.memory_limit_bytes == 0 and s.operator_form == 0


def test_create_fails_loudly_without_gpu(built):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(built.ProxSDPError) as e:
        built.Solver()
    assert e.value.code == -2  # PROXSDP_ERR_CUDA, no fallback
