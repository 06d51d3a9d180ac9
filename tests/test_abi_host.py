"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every entry point include/crkfr.h declares, rejects bad
configurations, and its host-computed reference element and CFL(N) agree
with the oracle (Sec. 2, Eq. soln.points; Sec. 5, under Eq. time.step.2d)."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

from paper_2512_08611_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def crk():
    B.build_library()
    from paper_2512_08611_gb300 import crkfr
    crkfr.lib()
    return crkfr


def declared_functions():
    text = open(os.path.join(ROOT, "include", "crkfr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(crkfr_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(crk):
    names = declared_functions()
    assert len(names) >= 15
    handle = ctypes.CDLL(B.library_path())
    for name in names:
        assert hasattr(handle, name), name
    # and the binding declares exactly these
    assert set(names) == set(crk.SIGNATURES)


def test_config_struct_layout(crk):
    assert ctypes.sizeof(crk.Config) == 64
    assert crk.Config.source.offset == 12
    assert crk.Config.gravity.offset == 16
    assert crk.Config.source_coef.offset == 40
    assert crk.Config.rk.offset == 48
    assert crk.Config.nc_face_mode.offset == 52
    assert crk.Config.coef_dissipation.offset == 56
    assert crk.Config.reserved.offset == 60


def test_scheme_switches_accept_only_the_built_readings(crk):
    """rk, nc_face_mode and coef_dissipation: the zero defaults and the
    explicit built values create a context; the other readings of the paper
    are refused with CRKFR_ERR_UNSUPPORTED and a reason, on every entry point
    that takes a config (contexts, ensembles, the allocation-free step)."""
    from paper_2512_08611_gb300.crkfr import Batch, CrkfrError, Solver
    for N in range(5):
        Solver("swe1d", N, rk=0)
        Solver("swe1d", N, rk=N + 1)
    Solver("swe1d", 2, source="chezy", source_coef=0.1, rk=3)
    Solver("swe2d", 3, nc_face="frozen", coef_dissipation=False)
    cases = [dict(rk=4, N=2), dict(rk=2, N=3), dict(rk=4, N=2, source="chezy", source_coef=0.1),
             dict(nc_face="literal", N=3), dict(nc_face="stagewise", N=3),
             dict(coef_dissipation=True, N=3)]
    for kw in cases:
        N = kw.pop("N")
        with pytest.raises(CrkfrError) as e:
            Solver("swe1d", N, **kw)
        assert e.value.status == -2, kw
        assert any(k in str(e.value) for k in ("rk", "nc_face_mode", "coef_dissipation")), str(e.value)
        with pytest.raises(CrkfrError) as e:
            Batch("swe1d", [(N, 10, 0.0, 1.0)], **kw)
        assert e.value.status == -2
    # values outside the enums and a non-zero reserved field are argument errors
    h = ctypes.c_void_p()
    for field, value in (("nc_face_mode", 7), ("coef_dissipation", 2), ("reserved", 1)):
        cfg = crk.make_config("swe1d", 2, "gl", 9.81, 0.5, 0.0, None, 0.0)
        setattr(cfg, field, value)
        assert crk.lib().crkfr_create(ctypes.byref(h), ctypes.byref(cfg)) == -1
        assert crk.lib().crkfr_last_error(None).decode() != ""
    # the allocation-free step checks the switches before touching the GPU
    cfg = crk.make_config("swe1d", 2, "gl", 9.81, 0.5, 0.0, None, 0.0, nc_face="literal")
    p = ctypes.c_void_p(16)
    assert crk.lib().crkfr_step_1d_noalloc(ctypes.byref(cfg), 10, 0.0, 1.0, p, p, p, 0.01, 1,
                                           None) == -2
    assert "nc_face_mode" in crk.lib().crkfr_last_error(None).decode()


def test_split_entry_points_refuse_contexts_they_do_not_serve(crk):
    """The limiter's and the adjoint's slab entry points and the record's
    halo blocks answer CRKFR_ERR_ARG for null arguments and
    CRKFR_ERR_STATE on a context that is not a 2D slab (no mesh here),
    before any GPU work."""
    from paper_2512_08611_gb300.crkfr import Solver
    s = Solver("swe2d", 2)
    L = crk.lib()
    ptrs = [ctypes.c_void_p() for _ in range(4)]
    refs = [ctypes.byref(x) for x in ptrs]
    cnt = ctypes.c_int64()
    fake = ctypes.c_void_p(16)
    assert L.crkfr_limiter_halo_buffers(None, 0, *refs, ctypes.byref(cnt)) == -1
    assert L.crkfr_limiter_halo_buffers(s.h, 0, *refs, ctypes.byref(cnt)) == -6
    assert L.crkfr_adjoint_halo_buffers(s.h, *refs, ctypes.byref(cnt)) == -6
    assert L.crkfr_record_halo_buffers(s.h, None, *refs, ctypes.byref(cnt)) == -1
    assert L.crkfr_record_halo_buffers(s.h, fake, *refs, ctypes.byref(cnt)) == -6
    assert L.crkfr_step_indicator(s.h, fake, None) == -6
    assert L.crkfr_adjoint_sums(s.h, fake, None) == -6
    assert L.crkfr_adjoint_local(s.h, fake, fake, 0.1, None) == -6
    assert L.crkfr_step_local_record(s.h, fake, 0.1, fake, 1, None) == -6
    assert all(p.value is None for p in ptrs)


def test_tile_size_setting(crk):
    """crkfr_set_tile_1d takes 0 (per mesh), 64, 96 or 128 threads on a 1D
    context; other values are argument errors, a 2D context refuses it."""
    from paper_2512_08611_gb300.crkfr import CrkfrError, Solver
    s = Solver("swe1d", 4)
    for t in (0, 64, 96, 128):
        s.set_tile_1d(t)
    for t in (32, 100, 256, -1):
        with pytest.raises(CrkfrError) as e:
            s.set_tile_1d(t)
        assert e.value.status == -1 and "threads" in str(e.value)
    with pytest.raises(CrkfrError) as e:
        Solver("swe2d", 3).set_tile_1d(96)
    assert e.value.status == -2


def test_only_periodic_meshes_are_built(crk):
    from paper_2512_08611_gb300.crkfr import CrkfrError, Solver
    s = Solver("swe2d", 2)
    for mask, status in ((0, -2), (1, -2), (2, -2), (4, -1), (-1, -1)):
        arr = (ctypes.c_int64 * 2)(4, 3)
        d2 = (ctypes.c_double * 2)
        assert crk.lib().crkfr_set_mesh(s.h, 2, arr, d2(0.0, 0.0), d2(1.0, 1.0), mask) == status
    with pytest.raises(CrkfrError) as e:
        Solver("swe1d", 2).set_mesh([5], [0.0], [1.0], periodic=False)
    assert e.value.status == -2 and "periodic" in str(e.value)


def test_bad_configs_are_rejected(crk):
    from paper_2512_08611_gb300.crkfr import CrkfrError, Solver
    with pytest.raises(CrkfrError) as e:
        Solver("swe1d", 5)
    assert e.value.status == -2
    with pytest.raises(CrkfrError):
        Solver("swe1d", 0, nodes="gll")
    with pytest.raises(CrkfrError):
        Solver("swe2d", 0)
    with pytest.raises(CrkfrError) as e:
        Solver("swe1d", 3, cfl_safety=1.5)
    assert e.value.status == -1
    with pytest.raises(CrkfrError):
        Solver("swe1d", 3, gravity=-1.0)


def test_bad_source_configs_are_rejected(crk):
    from paper_2512_08611_gb300.crkfr import Config, CrkfrError, Solver
    for system, source in (("varadv1d", "chezy"), ("swe1d", "linear"), ("swe2d", "linear")):
        with pytest.raises(CrkfrError) as e:
            Solver(system, 2, source=source, source_coef=1.0)
        assert e.value.status == -2
    for coef in (-1.0, float("inf"), float("nan")):
        with pytest.raises(CrkfrError) as e:
            Solver("swe1d", 2, source="chezy", source_coef=coef)
        assert e.value.status == -1
    h = ctypes.c_void_p()
    cfg = Config(1, 2, 0, 7, 9.81, 0.5, 0.0, 1.0, 0, 0, 0, 0)   # no such source
    assert crk.lib().crkfr_create(ctypes.byref(h), ctypes.byref(cfg)) == -1
    # a coefficient without a source is ignored
    Solver("swe1d", 2, source=None, source_coef=-5.0)


def test_calls_before_mesh_are_refused(crk):
    from paper_2512_08611_gb300.crkfr import CrkfrError, Solver
    s = Solver("swe1d", 2)
    with pytest.raises(CrkfrError) as e:
        s.time()
    assert e.value.status == -6


@pytest.mark.parametrize("N", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("family", ["gl", "gll"])
def test_nodes_and_cfl_match_oracle(crk, N, family):
    if family == "gll" and N == 0:
        pytest.skip("GLL needs N >= 1")
    from oracle.basis import Basis
    from paper_2512_08611_gb300.crkfr import Solver
    s = Solver("swe1d", N, nodes=family)
    xi, w = s.nodes()
    bs = Basis(N, family)
    assert np.max(np.abs(xi - bs.xi)) < 2e-16 * 4
    assert np.max(np.abs(w - bs.w)) < 2e-16 * 4
    with open(os.path.join(ROOT, "tests", "golden", "oracle_cfl.json")) as fh:
        want = json.load(fh)["cfl"][f"{N}_{family}"]
    assert s.cfl() == pytest.approx(want, rel=1e-8)


@pytest.mark.parametrize("N", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("family", ["gl", "gll"])
def test_imex_cfl_matches_oracle(crk, N, family):
    """With a source the CFL number is that of the explicit part of
    SSP3-IMEX(4,3,3) (stored by tests/golden/make_golden.py from the oracle)."""
    if family == "gll" and N == 0:
        pytest.skip("GLL needs N >= 1")
    from paper_2512_08611_gb300.crkfr import Solver
    with open(os.path.join(ROOT, "tests", "golden", "oracle_cfl.json")) as fh:
        want = json.load(fh)["cfl_imex"][f"{N}_{family}"]
    s = Solver("varadv1d", N, nodes=family, source="linear", source_coef=1.0)
    assert s.cfl() == pytest.approx(want, rel=1e-8)
    if N >= 1:
        s = Solver("swe2d", N, nodes=family, source="chezy", source_coef=0.01)
        assert s.cfl() == pytest.approx(want, rel=1e-8)


@pytest.mark.parametrize("system", ["swe1d_wb", "swe2d_wb"])
def test_well_balanced_systems_configure_like_standard(crk, system):
    """The well-balanced forms have the standard forms' variables, degrees,
    CFL numbers and sources."""
    from paper_2512_08611_gb300.crkfr import CrkfrError, Solver
    with open(os.path.join(ROOT, "tests", "golden", "oracle_cfl.json")) as fh:
        g = json.load(fh)
    for N in (1, 3):
        assert Solver(system, N).cfl() == pytest.approx(g["cfl"][f"{N}_gl"], rel=1e-8)
        s = Solver(system, N, source="chezy", source_coef=0.1)
        assert s.cfl() == pytest.approx(g["cfl_imex"][f"{N}_gl"], rel=1e-8)
    with pytest.raises(CrkfrError) as e:
        Solver(system, 2, source="linear", source_coef=1.0)
    assert e.value.status == -2
    if system == "swe2d_wb":
        with pytest.raises(CrkfrError):
            Solver(system, 0)
    with pytest.raises(CrkfrError) as e:
        Solver(system, 2, gravity=0.0)
    assert e.value.status == -1


def test_explicit_cfl_number_is_used(crk):
    from paper_2512_08611_gb300.crkfr import Solver
    assert Solver("swe1d", 3, cfl_number=0.05).cfl() == 0.05


def test_fp64_probe_refuses_bad_arguments_without_a_launch(crk):
    """Out-of-range modes, grid or loop sizes and null pointers return
    CRKFR_ERR_ARG before any CUDA call (runs without a GPU)."""
    L = crk.lib()
    f = ctypes.c_double(-1.0)
    sink = ctypes.c_void_p(16)   # never dereferenced: the checks come first
    for mode, blocks, iters in ((3, 1, 1), (-1, 1, 1), (0, 0, 1), (0, 9729, 1), (0, 1, 0),
                                (0, 1, 65537)):
        assert L.crkfr_fp64_probe(mode, blocks, iters, sink, ctypes.byref(f), None) == -1
    assert L.crkfr_fp64_probe(0, 1, 1, None, ctypes.byref(f), None) == -1
    assert L.crkfr_fp64_probe(0, 1, 1, sink, None, None) == -1
