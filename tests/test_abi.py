"""Host-side checks of the C ABI (no GPU needed).

The library must build for sm_103a, load, export every entry point that
include/*.h declares, agree with the Python binding on the layout of
lbm_ace_params, and reject invalid parameters before touching the device.
"""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2203_05230_gb300 import lbm_ace as A

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(lbm_ace_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_function():
    L = A.load()
    names = declared_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(A.EXPORTS) <= set(names)
    out = subprocess.run(["nm", "-D", "--defined-only", A.library_path()], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}\b", out), n


def test_params_struct_layout_matches_header(tmp_path):
    fields = [f for f, _ in A.lbm_ace_params._fields_]
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbm_ace.h"', "int main(void){",
           'printf("%zu\\n", sizeof(lbm_ace_params));']
    for f in fields:
        src.append(f'printf("%zu\\n", offsetof(lbm_ace_params, {f}));')
    src.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(A.lbm_ace_params)
    for f, off in zip(fields, vals[1:]):
        assert getattr(A.lbm_ace_params, f).offset == off, f


def test_defaults_are_the_64x64_vortex():
    p = A.params_default()
    assert (p.nx, p.ny, p.tau, p.eps, p.U0, p.T_period) == (64, 64, 0.8, 1.0, 0.04, 2000.0)
    assert (p.xc, p.yc, p.R, p.vortex_sign, p.M) == (32.0, 48.0, 9.6, -1.0, -1.0)
    assert A.status_string(A.EINVAL) == "invalid argument"


@pytest.mark.parametrize("kw,frag", [
    (dict(nx=2), "must be >= 3"),
    (dict(ny=1), "must be >= 3"),
    (dict(tau=0.5), "tau"),
    (dict(tau=float("nan")), "tau"),
    (dict(eps=0.0), "eps"),
    (dict(M=0.2), "differs from c_s^2"),
    (dict(precision=7), "precision"),
    (dict(model=5), "model"),
    (dict(velocity_kind=9), "velocity kind"),
    (dict(T_period=0.0), "T_period"),
    (dict(velocity_kind=A.VEL_FIELD), "velocity field"),
    (dict(rows_per_cta=-1), "rows_per_cta"),
    (dict(kernel_variant=5), "kernel_variant"),
    (dict(nx=65, kernel_variant=4), "even nx"),
    (dict(nx=66, precision=1, kernel_variant=2), "multiple of 16"),
    (dict(nx=67, precision=0, kernel_variant=2), "multiple of 16"),
])
def test_invalid_parameters_are_rejected_on_the_host(kw, frag):
    with pytest.raises(A.LbmAceError) as e:
        A.Lattice(**kw)
    assert e.value.status == A.EINVAL
    assert frag in str(e.value)


def test_non_finite_phi0_is_rejected():
    phi0 = np.full((8, 8), 0.5)
    phi0[3, 4] = np.nan
    with pytest.raises(A.LbmAceError) as e:
        A.Lattice(nx=8, ny=8, phi0=phi0)
    assert e.value.status == A.EINVAL and "phi0[28]" in str(e.value)


@pytest.mark.parametrize("precision", [1, 2, 3])
def test_phi0_beyond_fp32_range_is_rejected_for_fp32_storage(precision):
    """The FP32-based forms keep phi in FP32: a value that rounds to infinity there
    (|v| >= 2^128 - 2^103) is rejected before any device work; one just below is not."""
    phi0 = np.full((8, 8), 0.5)
    phi0[2, 5] = -(2.0 ** 128 - 2.0 ** 103)
    with pytest.raises(A.LbmAceError) as e:
        A.Lattice(nx=8, ny=8, phi0=phi0, precision=precision)
    assert e.value.status == A.EINVAL and "phi0[21] is not finite as FP32" in str(e.value)
    phi0[2, 5] = -np.nextafter(2.0 ** 128 - 2.0 ** 103, 0.0)  # rounds to -FLT_MAX
    assert np.isfinite(np.float32(phi0[2, 5]))
    for p in (precision, 0):  # and FP64 storage takes any finite value
        try:
            A.Lattice(nx=8, ny=8, phi0=phi0 if p else np.where(phi0 == 0.5, 0.5, -1e300), precision=p)
        except A.LbmAceError as e:
            assert e.status in (A.ECUDA, A.ENOMEM), e


def test_consistent_mobility_is_accepted_by_validation():
    """M = c_s^2 (tau - 1/2) passes validation (it then fails only for want of a GPU here)."""
    try:
        A.Lattice(nx=8, ny=8, tau=0.8, M=0.1)
    except A.LbmAceError as e:
        assert e.status in (A.ECUDA, A.ENOMEM), e


def test_hybrid_stats_layout_matches_header(tmp_path):
    fields = [f for f, _ in A.lbm_ace_hybrid_stats._fields_]
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbm_ace_surrogate.h"', "int main(void){",
           'printf("%zu\\n", sizeof(lbm_ace_hybrid_stats));',
           'printf("%d %d %d\\n", LBM_ACE_NET_WIDTH, LBM_ACE_NET_K, LBM_ACE_NET_PARAMS);']
    for f in fields:
        src.append(f'printf("%zu\\n", offsetof(lbm_ace_hybrid_stats, {f}));')
    src.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(A.lbm_ace_hybrid_stats)
    assert vals[1:4] == [A.NET_WIDTH, A.NET_K, A.NET_PARAMS]
    for f, off in zip(fields, vals[4:]):
        assert getattr(A.lbm_ace_hybrid_stats, f).offset == off, f


def test_net_parameter_count_matches_the_oracle():
    from oracle import surrogate as S
    assert S.param_count() == A.NET_PARAMS
    assert S.K_STEPS == A.NET_K and S.WIDTHS[1] == A.NET_WIDTH


def test_net_entry_points_reject_null_handles():
    L = A.load()
    assert L.lbm_ace_net_set_params(None, None, 0) == A.EINVAL
    assert L.lbm_ace_net_forward(None, None, None, None, None, 1, 8, 8) == A.EINVAL
    assert L.lbm_ace_hybrid_advance(None, None, 1, 1e-6, 0.1, None) == A.EINVAL
    assert L.lbm_ace_get_phi_device(None, None) == A.EINVAL
    assert b"NULL" in L.lbm_ace_net_last_error(None)
