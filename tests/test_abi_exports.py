"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/pbit.h; the binding's struct layouts match the C
compiler's (no compute call is made: no GPU here)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pbit.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pb_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2510_23419_gb300 import _build
    return ctypes.CDLL(_build.build())


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2510_23419_gb300 import native
    for n in _declared():
        assert hasattr(native, n), n


def test_struct_layouts_match_c(tmp_path):
    from paper_2510_23419_gb300 import native
    prog = tmp_path / "sz.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "pbit.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(pb_instance_desc), offsetof(pb_instance_desc, J), offsetof(pb_instance_desc, colour), 0);
  printf("%zu %zu %zu %zu\n", sizeof(pb_schedule), offsetof(pb_schedule, beta0), offsetof(pb_schedule, betas), 0);
  printf("%zu %zu %zu %zu\n", sizeof(pb_anneal_opts), offsetof(pb_anneal_opts, target_energy), 0, 0);
  printf("%zu %zu %zu %zu\n", sizeof(pb_tune_result), offsetof(pb_tune_result, candidate_wt), offsetof(pb_tune_result, probe_ms), 0);
  printf("%zu %zu %zu %zu\n", sizeof(pb_server_opts), offsetof(pb_server_opts, gather_us), 0, 0);
  printf("%zu %zu %zu %zu\n", sizeof(pb_server_stats), offsetof(pb_server_stats, rounds), offsetof(pb_server_stats, max_ms), 0);
  return 0; }''')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    rows = [list(map(int, l.split())) for l in subprocess.check_output([str(exe)]).decode().split("\n") if l]
    D, S, O = native.pb_instance_desc, native.pb_schedule, native.pb_anneal_opts
    assert rows[0][:3] == [ctypes.sizeof(D), D.J.offset, D.colour.offset]
    assert rows[1][:3] == [ctypes.sizeof(S), S.beta0.offset, S.betas.offset]
    assert rows[2][:2] == [ctypes.sizeof(O), O.target_energy.offset]
    T, SO, SS = native.pb_tune_result, native.pb_server_opts, native.pb_server_stats
    assert rows[3][:3] == [ctypes.sizeof(T), T.candidate_wt.offset, T.probe_ms.offset]
    assert rows[4][:2] == [ctypes.sizeof(SO), SO.gather_us.offset]
    assert rows[5][:3] == [ctypes.sizeof(SS), SS.rounds.offset, SS.max_ms.offset]


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2510_23419_gb300 import _build, native
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "absent.so"))
    monkeypatch.setattr(native, "_lib", None)
    with pytest.raises(RuntimeError, match="CUDA library missing"):
        native.load()
