"""Host-side checks of the C ABI: the library builds, loads and exports every
function include/htd.h declares; the ctypes structs match the C layout; the
host-only parameter selection (htd_plan) agrees with the oracle and rejects bad
input.  No CUDA compute call is made here."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
from paper_2006_16861_gb300 import htd
from paper_2006_16861_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "htd.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(htd_[A-Za-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    lib = htd.load()
    names = declared_functions()
    assert set(names) == set(htd.EXPORTS)
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", htd.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (htd_\w+)", out))
    assert set(names) <= exported


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "htd.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(htd_grid),"
        " sizeof(htd_options), sizeof(htd_params), sizeof(htd_solve_info),"
        " offsetof(htd_solve_info, hist), offsetof(htd_params, nP), offsetof(htd_options, damping),"
        " offsetof(htd_options, stencil_a), offsetof(htd_options, stencil_gamma),"
        " offsetof(htd_options, tblock));"
        "printf(\"%zu %zu %zu %zu %zu\\n\", offsetof(htd_options, s3_kernel),"
        " offsetof(htd_options, launch), offsetof(htd_options, wait_limit_ns),"
        " offsetof(htd_options, s3_rhs_per_cta), offsetof(htd_params, rhs_per_cta));"
        "return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [ctypes.sizeof(htd.Grid), ctypes.sizeof(htd.Options), ctypes.sizeof(htd.Params),
            ctypes.sizeof(htd.SolveInfo), htd.SolveInfo.hist.offset, htd.Params.nP.offset,
            htd.Options.damping.offset, htd.Options.stencil_a.offset,
            htd.Options.stencil_gamma.offset, htd.Options.tblock.offset,
            htd.Options.s3_kernel.offset, htd.Options.launch.offset,
            htd.Options.wait_limit_ns.offset, htd.Options.s3_rhs_per_cta.offset,
            htd.Params.rhs_per_cta.offset]
    assert got == want


@pytest.mark.parametrize("field,value", [("tb_rows", 7), ("tb_rows", -1), ("tb_form", 5),
                                         ("tb_form", -1), ("s3_kernel", 5), ("s3_kernel", -1),
                                         ("s3_stages", 3), ("s3_stages", 8), ("s3_zchunk", -1),
                                         ("launch", 8), ("wait_limit_ns", -1),
                                         ("s3_rhs_per_cta", 3), ("s3_rhs_per_cta", -1)])
def test_plan_rejects_bad_kernel_selection(field, value):
    """The kernel-selection fields of htd_options are validated on the host,
    like every other option (HTD_ERR_ARG)."""
    p = W.config_2d_constant(21)
    htd.plan(p)                                       # the defaults are accepted
    with pytest.raises(htd.HtdError) as e:
        htd.plan(p, **{field: value})
    assert e.value.status == 1


def test_plan_accepts_every_documented_kernel_selection():
    p = W.config_2d_constant(21)
    for kw in (dict(tb_rows=8, tb_form=htd.TB_PAIR_SD), dict(tb_form=htd.TB_COLUMN),
               dict(tb_form=htd.TB_RESIDENT),
               dict(s3_kernel=htd.S3_NODE_128x2, s3_stages=7, s3_zchunk=16),
               dict(s3_kernel=htd.S3_ZMARCH),
               dict(launch=htd.LAUNCH_NO_OVERLAP | htd.LAUNCH_NO_GRAPH),
               dict(wait_limit_ns=1000)):
        assert htd.plan(p, **kw)["nP"] > 0


def test_default_options():
    o = htd.htd_default_options()
    assert (o.precision, o.mode, o.krylov, o.T, o.rho, o.nP, o.stencil, o.restart,
            o.max_rhs, o.proj_periods, o.integrator, o.damping, o.stencil_a, o.stencil_gamma,
            o.tblock) == \
        (htd.FP64, htd.MODE_TABLE1, htd.FGMRES, 10, 0.25, 0, htd.STENCIL_Q1MIX, 20, 1, 1,
         htd.ACD, htd.DAMP_NODE, 0.5, 1.0, 0)


PROBLEMS = [
    lambda: W.config_2d_constant(101),
    lambda: W.config_2d_constant(57, ppw=6.0, layer=8, T=3),
    lambda: W.config_2d_heterogeneous(201, layer=10, T=5),
    lambda: W.config_3d_layered(20, layer=4, T=2),
]


STENCILS = [("q1mix", {}), ("fd5", {}), ("family", {"stencil_a": 0.3, "stencil_gamma": 0.6}),
            ("family", {"stencil_a": 1.0, "stencil_gamma": 0.0})]


@pytest.mark.parametrize("mk", PROBLEMS)
@pytest.mark.parametrize("stencil,kw", STENCILS, ids=["q1mix", "fd5", "family", "family_a1g0"])
def test_plan_matches_oracle_parameters(mk, stencil, kw):
    p = mk()
    mine = htd.plan(p, stencil=stencil, **kw)
    ref = oracle.Oracle(p, stencil, **kw).param_dict()
    assert mine["nP"] == ref["nP"]
    assert mine["T"] == ref["T"] and mine["steps"] == ref["nsteps"]
    for a, b in [("omega_c", "omega"), ("k_min", "k_min"), ("k_max", "k_max"),
                 ("lam_max_reH", "lam_max_reH"), ("lam_max_A", "lam_max_A"), ("dt", "dt"),
                 ("alpha", "alpha"), ("beta", "beta"), ("rho", "rho")]:
        assert mine[a] == pytest.approx(ref[b], rel=1e-12), a


def test_plan_rejects_bad_input():
    p = W.config_2d_constant(31, T=2)
    ok = htd.plan(p)
    with pytest.raises(htd.HtdError) as e:
        htd.plan(p, nP=ok["nP"] - 4)               # violates the CFL bound
    assert e.value.status == 4
    with pytest.raises(htd.HtdError) as e:
        htd.plan(p, nP=ok["nP"] + 2)               # not a multiple of 4
    assert e.value.status == 4
    c = p.c_cell.copy()
    c[3, 4] = np.nan
    with pytest.raises(htd.HtdError) as e:
        htd.htd_plan(2, p.n, p.h, c, p.R_node, p.omega, 0, htd.make_options(p))
    assert e.value.status == 5
    c[3, 4] = -1.0
    with pytest.raises(htd.HtdError) as e:
        htd.htd_plan(2, p.n, p.h, c, p.R_node, p.omega, 0, htd.make_options(p))
    assert e.value.status == 1
    R = p.R_node.copy()
    R[0, 0] = -1
    with pytest.raises(htd.HtdError) as e:
        htd.htd_plan(2, p.n, p.h, p.c_cell, R, p.omega, 0, htd.make_options(p))
    assert e.value.status == 1
    for kw in ({"restart": 0}, {"restart": 65}, {"T": 0}, {"rho": 1.5}, {"max_rhs": -1},
               {"max_rhs": 257}, {"mode": "project", "proj_periods": 3},
               {"mode": "project", "proj_periods": -1}, {"damping": "cell"},
               {"stencil": "family", "stencil_a": -0.1}, {"stencil": "family", "stencil_a": 1.5},
               {"stencil": "family", "stencil_gamma": float("nan")},
               {"stencil": "family", "stencil_gamma": 2.0}, {"tblock": 2}, {"tblock": -1}):
        with pytest.raises(htd.HtdError) as e:
            htd.plan(p, **kw)
        assert e.value.status == 1
    with pytest.raises(htd.HtdError):
        htd.htd_plan(2, p.n, -1.0, p.c_cell, p.R_node, p.omega, 0, htd.make_options(p))
    with pytest.raises(htd.HtdError):
        htd.htd_plan(4, p.n, p.h, p.c_cell, p.R_node, p.omega, 0, htd.make_options(p))
    with pytest.raises(htd.HtdError):
        htd.htd_plan(2, p.n, p.h, p.c_cell, p.R_node, p.omega, 1, htd.make_options(p))
    o = htd.make_options(p)
    o.stencil = 3
    with pytest.raises(htd.HtdError) as e:
        htd.htd_plan(2, p.n, p.h, p.c_cell, p.R_node, p.omega, 0, o)
    assert e.value.status == 1
    # the family's weights are read only for HTD_STENCIL_FAMILY
    assert htd.plan(p, stencil="q1mix", stencil_a=7.0)["nP"] == ok["nP"]


@pytest.mark.parametrize("d", [2, 3])
def test_family_corners_are_q1mix_and_fd5(d):
    """FAMILY(0.5, 1) plans exactly like Q1MIX and FAMILY(0, 0) like FD5."""
    p = W.config_2d_constant(41, T=2) if d == 2 else W.config_3d_layered(12, layer=3, T=2)
    for st, a, g in (("q1mix", 0.5, 1.0), ("fd5", 0.0, 0.0)):
        assert htd.plan(p, stencil="family", stencil_a=a, stencil_gamma=g) == htd.plan(p, stencil=st)


def test_status_strings():
    for s in range(9):
        assert htd.htd_status_string(s)


@pytest.mark.parametrize("damping", ["node", "cell"])
def test_plan_abd_matches_oracle(damping):
    """The backward-differences parameters of Sec. 6.1 (omega above k_max, n_P, dt)
    agree with the oracle's; the admissible damping is weaker than for I_acd."""
    p = W.config_2d_constant(41, ppw=8.0, layer=6, T=3)
    p = W.Problem(p.name, p.ndim, p.n, p.h, p.c_cell, 0.5 * p.R_node, p.omega, p.F, p.T, p.rho)
    got = htd.plan(p, integrator="abd", damping=damping)
    o = oracle.Oracle(p, integrator="abd", damping=damping)
    assert got["nP"] == o.params.nP
    assert got["omega_c"] == pytest.approx(o.params.omega, rel=1e-14)
    assert got["dt"] == pytest.approx(o.params.dt, rel=1e-14)
    assert got["omega_c"] > got["k_max"]
    # R0 = 2 omega at c_min = 1 sits at the limit 2 lambda_max(Im H) / k_max^2 -> 4
    q = W.config_2d_constant(41, ppw=8.0, layer=6, T=3)
    with pytest.raises(htd.HtdError) as e:
        htd.plan(q, integrator="abd")
    assert e.value.status == 4


@pytest.mark.parametrize("damping", ["node", "cell"])
@pytest.mark.parametrize("a,g", [(0.3, 0.6), (1.0, 0.0)])
def test_plan_abd_family_matches_oracle(damping, a, g):
    """I_abd's parameters with a stencil-family member agree with the oracle's."""
    p = W.config_2d_constant(41, ppw=8.0, layer=6, T=3)
    p = W.Problem(p.name, p.ndim, p.n, p.h, p.c_cell, 0.5 * p.R_node, p.omega, p.F, p.T, p.rho)
    got = htd.plan(p, integrator="abd", damping=damping, stencil="family", stencil_a=a,
                   stencil_gamma=g)
    o = oracle.Oracle(p, integrator="abd", damping=damping, stencil="family", stencil_a=a,
                      stencil_gamma=g)
    assert got["nP"] == o.params.nP
    assert got["omega_c"] == pytest.approx(o.params.omega, rel=1e-14)
    assert got["lam_max_reH"] == pytest.approx(o.params.lam_max_reH, rel=1e-12)


def test_plan_rejects_empty_and_oversized_grids():
    """n[a] = 0 (an empty grid) and more than 2^24 nodes on an axis are refused
    before any array is read; a 1 x 1 grid is accepted."""
    c = np.ones((2, 2))
    R = np.zeros((1, 1))
    assert htd.htd_plan(2, (1, 1), 0.1, c, R, 5.0, 0, htd.make_options(T=2, rho=0.25))["nP"] > 0
    for n in ((0, 5), (5, 0), (1 << 25, 1)):
        with pytest.raises(htd.HtdError) as e:
            htd.htd_plan(2, n, 0.1, np.ones(1), np.ones(1), 5.0, 0, htd.make_options(T=2, rho=0.25))
        assert e.value.status == 1
    # each axis within 2^24 but the product beyond the 2^34-node limit: refused
    # before the product is formed (2^72 would wrap an int64 to 0) and before
    # the one-element arrays are read
    for n in ((1 << 24, 1 << 24, 1 << 24), (1 << 24, 1 << 24, 1 << 16), (1 << 24, 1 << 11, 1)):
        with pytest.raises(htd.HtdError) as e:
            htd.htd_plan(3, n, 0.1, np.ones(1), np.ones(1), 5.0, 0, htd.make_options(T=2, rho=0.25))
        assert e.value.status == 1
