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
    assert ctypes.sizeof(crk.Config) == 48
    assert crk.Config.source.offset == 12
    assert crk.Config.gravity.offset == 16
    assert crk.Config.source_coef.offset == 40


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
    cfg = Config(1, 2, 0, 7, 9.81, 0.5, 0.0, 1.0)   # no such source
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
