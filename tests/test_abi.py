"""The C-ABI library builds, loads and exports every entry point include/*.h
declares; host-side argument checks work without a GPU (no compute calls)."""
import ctypes
import glob
import os
import re

import numpy as np

import pytest

from conftest import ROOT


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(lbm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1203_6350_gb300 import lbm

    return lbm.load()


def test_headers_declare_the_boundary():
    names = _declared()
    for n in ("lbm_create", "lbm_set_sponge", "lbm_step", "lbm_moments", "lbm_destroy",
              "lbm_init_equilibrium", "lbm_diagnostics", "lbm_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in sorted(_declared()):
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_1203_6350_gb300 import lbm

    bound = {s[0] for s in lbm.SIGNATURES}
    assert _declared() <= bound, _declared() - bound
    for n in _declared():
        assert callable(getattr(lbm, n)), n


def test_version_string(lib):
    from paper_1203_6350_gb300 import lbm

    assert "D2Q9" in lbm.lbm_version()


@pytest.mark.parametrize("kw,frag", [
    (dict(nx=0), "size"),
    (dict(ny=-3), "size"),
    (dict(storage=7), "storage"),
    (dict(bc=5), "bc"),
    (dict(rho0=0.0), "rho0"),
    (dict(rho0=float("nan")), "rho0"),
    (dict(rates_s=float("inf")), "rate"),
    (dict(n=-1.0), "Guo"),
])
def test_create_rejects_bad_arguments_before_touching_the_device(lib, kw, frag):
    from paper_1203_6350_gb300 import lbm

    args = dict(nx=16, ny=8, storage=1, rho0=1.0, bc=0, rates_s=1.9, n=0.5)
    args.update(kw)
    rates = lbm.make_rates(args["rates_s"], args["n"], 0.5)
    rc, h = lbm.lbm_create(args["nx"], args["ny"], args["storage"], args["rho0"], 0.0, 0.0, rates,
                           args["bc"])
    assert rc == lbm.LBM_ERR_ARG
    assert not h.value
    assert frag in lbm.lbm_last_error(None)


def test_null_handle_calls_are_argument_errors(lib):
    from paper_1203_6350_gb300 import lbm

    assert lbm.lbm_step(None, 1) == lbm.LBM_ERR_ARG
    assert lbm.lbm_moments(None, None, None, None, 0) == lbm.LBM_ERR_ARG
    assert lbm.lbm_diagnostics(None, 0, 0, 1, 1, None) == lbm.LBM_ERR_ARG
    assert lbm.lbm_state_bytes(None) == 0
    assert lbm.lbm_time(None) == -1
    lbm.lbm_destroy(None)


def test_rates_struct_layout_matches_header():
    from paper_1203_6350_gb300 import lbm

    assert ctypes.sizeof(lbm.lbm_rates) == 11 * 8
    assert ctypes.sizeof(lbm.lbm_allocator) == 3 * ctypes.sizeof(ctypes.c_void_p)


def test_autotuner_configurations_cover_every_batched_kernel():
    from paper_1203_6350_gb300 import autotune

    f32 = autotune.configurations("f32")
    kernels = {(c, s) for c, s, _, _ in f32}
    assert kernels == {(1, 1), (2, 1), (2, 2)}
    assert [t for c, s, *t in f32 if s == 2] == [list(autotune.TWO_STEP_TILE)]
    assert {(c, s) for c, s, _, _ in autotune.configurations("f64")} == {(1, 1)}
    # the signature ignores order and buckets sizes by powers of two
    assert autotune.signature([(100, 60), (64, 33)]) == autotune.signature([(70, 40), (127, 63)])


def test_stability_map_calls_check_arguments_before_touching_the_device(lib):
    """lbm_vn_growth / lbm_vn_chi_crit validate every argument on the host; an
    empty case list is a no-op.  None of these reach the device."""
    from paper_1203_6350_gb300 import lbm, stability

    assert lbm.LBM_VN_FIELDS == len(stability.FIELDS) == 15
    with open(os.path.join(ROOT, "include", "lbm.h")) as fh:
        assert "#define LBM_VN_FIELDS 15" in fh.read()
    good = stability.case(1.9, chi=0.5)
    v = np.array([2], dtype=np.int32)
    out = np.zeros(1)

    def growth(variant=v, cases=good, n=1, nk=8, prec=0, dst=out):
        c = np.ascontiguousarray(cases, dtype=np.float64)
        return lbm.lbm_vn_growth(variant.ctypes.data, c.ctypes.data, n, nk, prec,
                                 None if dst is None else dst.ctypes.data, None, None)

    def crit(lo=0.0, hi=8.0, nscan=17, iters=40, tol=1e-9, n=1):
        return lbm.lbm_vn_chi_crit(v.ctypes.data, good.ctypes.data, n, 8, 0, lo, hi, nscan, iters,
                                   tol, out.ctypes.data, None)

    assert growth(n=0) == lbm.LBM_OK and crit(n=0) == lbm.LBM_OK
    assert growth(variant=np.array([4], dtype=np.int32)) == lbm.LBM_ERR_ARG  # viscosity sponge
    assert "variant" in lbm.lbm_vn_last_error()
    assert growth(variant=np.array([-1], dtype=np.int32)) == lbm.LBM_ERR_ARG
    bad = good.copy()
    bad[3] = np.nan
    assert growth(cases=bad) == lbm.LBM_ERR_ARG
    bad = good.copy()
    bad[14] = -0.1
    assert growth(cases=bad) == lbm.LBM_ERR_ARG
    assert growth(nk=-1) == lbm.LBM_ERR_ARG
    assert growth(prec=2) == lbm.LBM_ERR_ARG  # FP16 is not a precision of the map
    assert growth(dst=None) == lbm.LBM_ERR_ARG
    assert growth(n=-1) == lbm.LBM_ERR_ARG
    assert crit(nscan=1) == lbm.LBM_ERR_ARG
    assert crit(lo=1.0, hi=1.0) == lbm.LBM_ERR_ARG
    assert crit(lo=-0.5) == lbm.LBM_ERR_ARG
    assert crit(iters=201) == lbm.LBM_ERR_ARG
    assert crit(tol=float("nan")) == lbm.LBM_ERR_ARG
    # host-side marshalling
    vv, cc = stability._marshal(["I", "III"], np.stack([good, good]))
    assert vv.tolist() == [1, 3] and cc.shape == (2, 15)
    with pytest.raises(ValueError):
        stability._marshal("II", np.zeros((1, 14)))
    np.testing.assert_array_equal(stability.case([1.0] * 3 + [1.5] * 6, 0.2, 0.3, 0.4, (0.1, -0.1),
                                                 0.7),
                                  [1, 1, 1, 1.5, 1.5, 1.5, 1.5, 1.5, 1.5, 0.3, 0.4, 0.1, -0.1, 0.7,
                                   0.2])


@pytest.mark.parametrize("kw,frag", [
    (dict(nx=0), "sizes"),
    (dict(nz=70000), "65535"),
    (dict(storage=2), "storage"),
    (dict(bc=2), "bc"),
    (dict(rho0=0.0), "rho0"),
    (dict(s=float("nan")), "rates"),
    (dict(n=-0.5), "Guo"),
])
def test_lbm3_create_rejects_bad_arguments_before_touching_the_device(lib, kw, frag):
    from paper_1203_6350_gb300 import lbm

    a = dict(nx=8, ny=8, nz=8, storage=1, rho0=1.0, s=1.9, n=0.5, bc=0)
    a.update(kw)
    s15 = np.full(15, a["s"])
    rc, h = lbm.lbm3_create(a["nx"], a["ny"], a["nz"], a["storage"], a["rho0"], (0.0, 0.0, 0.0),
                            s15.ctypes.data, a["n"], 0.5, a["bc"])
    assert rc == lbm.LBM_ERR_ARG
    assert not h.value
    assert frag in lbm.lbm3_last_error(None)


def test_lbm3_null_handle_calls_are_argument_errors(lib):
    from paper_1203_6350_gb300 import lbm

    assert lbm.lbm3_step(None, 1) == lbm.LBM_ERR_ARG
    assert lbm.lbm3_moments(None, None, None, None, None) == lbm.LBM_ERR_ARG
    assert lbm.lbm3_init_equilibrium(None, None, None, None, None) == lbm.LBM_ERR_ARG
    assert lbm.lbm3_set_sponge(None, 2, None, None, None, 1.0, (0, 0, 0)) == lbm.LBM_ERR_ARG
    assert lbm.lbm3_time(None) == -1
    lbm.lbm3_destroy(None)


def test_header_is_c99_and_links_from_plain_c(lib, tmp_path):
    """The boundary is usable from C: include/lbm.h compiles as strict C99,
    a C program links against liblbm.so, reads the version and gets
    LBM_ERR_ARG (nothing done, no device touched) for NULL handles."""
    import shutil
    import subprocess

    from paper_1203_6350_gb300 import build

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "lbm.h"
int main(void) {
    const char* v = lbm_version();
    if (!v || !strlen(v)) return 1;
    if (lbm_step(NULL, 1) != LBM_ERR_ARG) return 2;
    if (lbm_moments(NULL, NULL, NULL, NULL, 0) != LBM_ERR_ARG) return 3;
    if (lbm_batch_step(NULL, 1) != LBM_ERR_ARG) return 4;
    if (lbm3_step(NULL, 1) != LBM_ERR_ARG) return 5;
    if (lbm_batch_state_bytes(NULL, 0) != 0) return 6;
    printf("%s\n", v);
    return 0;
}
''')
    exe = tmp_path / "abi"
    inc = os.path.join(ROOT, "include")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc,
                        str(src), "-L", build.BUILD, "-llbm", "-Wl,-rpath," + build.BUILD,
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert r.stdout.strip()


def test_arithmetic_property_reads_the_mode_without_a_warning(lib, monkeypatch):
    """Lattice.arithmetic turns lbm_get_arithmetic's non-negative return into the
    mode's name (1 is "compensated", not a warning code) and raises on an error."""
    import warnings

    from paper_1203_6350_gb300 import lbm

    lat = object.__new__(lbm.Lattice)
    lat.h = None
    for code, name in lbm.ARITHMETIC_NAMES.items():
        monkeypatch.setattr(lbm, "lbm_get_arithmetic", lambda h, c=code: c)
        with warnings.catch_warnings():
            warnings.simplefilter("error")
            assert lat.arithmetic == name
    monkeypatch.setattr(lbm, "lbm_get_arithmetic", lambda h: lbm.LBM_ERR_ARG)
    with pytest.raises(lbm.LbmError):
        _ = lat.arithmetic
    lat.h = None  # nothing to close
