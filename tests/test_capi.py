"""The C-ABI library loads, exports every entry point of include/spmc.h and
rejects invalid plans before touching the GPU.  CPU only."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "spmc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spmc_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2608_22190_b300 import build as B
    B.build()
    from paper_2608_22190_b300 import _lib as L
    syms = declared_symbols()
    assert len(syms) >= 12
    for s in syms:
        assert hasattr(L.lib, s), s
    assert sorted(L.exported_symbols()) == syms


def test_invalid_plans_rejected_without_gpu():
    from paper_2608_22190_b300 import _lib as L

    def mk(**kw):
        d = L.PlanDesc()
        base = dict(dim=1, n_space=8, time_family=0, max_intervals=1, max_degree=4, M=64, K=1, tol=0.0,
                    n_ref=10, n_sub=4, shell=1e-4, max_steps=64, kappa=1.0, seed=0, precision=0, batch=1,
                    walk_mode=0)
        base.update(kw)
        for k, v in base.items():
            setattr(d, k, v)
        return d

    h = C.c_void_p()
    for bad in [dict(dim=0), dict(dim=6), dict(n_space=1), dict(n_space=40), dict(M=0), dict(K=0),
                dict(n_sub=3), dict(n_sub=32), dict(kappa=0.0), dict(shell=-1.0), dict(shell=0.5), dict(batch=0),
                dict(time_family=2), dict(precision=5), dict(max_degree=0), dict(walk_mode=2),
                dict(walk_mode=-1)]:
        assert L.lib.spmc_plan(C.byref(mk(**bad)), C.byref(h)) == L.SPMC_ERR_INVALID, bad
        assert not h.value
    assert L.lib.spmc_plan(None, C.byref(h)) == L.SPMC_ERR_INVALID
    assert L.lib.spmc_version().startswith(b"spmc-b300")


def test_walk_division_by_invariant_integers(tmp_path):
    """The walk splits walk ids with a multiply-shift quotient (FastDiv,
    Granlund-Montgomery); built by nvcc for the host and run on the host
    cores, it equals the integer quotient for every divisor below 4096 on
    every numerator below 2^16 and at the top of the 32-bit range, and for
    random divisors of every bit length next to multiples of the divisor."""
    import shutil
    import subprocess
    nvcc = os.environ.get("NVCC", "nvcc")
    if shutil.which(nvcc) is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "fastdiv_check")
    src = os.path.join(ROOT, "tests", "fastdiv_host_check.cu")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-o", exe, src],
                   check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 wrong" in r.stdout
