"""CPU checks of the C ABI: the library builds and loads, exports every entry
point include/st.h declares, and its host-side setup (collocation nodes, Q,
eigen-decomposition, time transfers, level planning) matches the oracle.  No
GPU work is launched."""
import os
import re

import numpy as np
import pytest

from oracle import collocation as col

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def stlib():
    from paper_2006_12883_gb300 import build, stlib as s
    build()
    return s


def _declared_symbols():
    with open(os.path.join(ROOT, "include", "st.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(st_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(stlib):
    L = stlib.lib()
    names = _declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(stlib._SIGS), set(names) - set(stlib._SIGS)


def test_solver_opts_layout_and_defaults(stlib):
    """The binding's st_solver_opts matches the C struct: the library's
    defaults land in the fields the header documents, through the last one
    (a field missing or out of order in the binding would shift them)."""
    C_FIELDS = [n.strip() for decl in re.findall(r"\b(?:int|double)\s+([^;]+);", _struct_text("st_solver_opts"))
                for n in decl.split(",")]
    assert [f for f, _ in stlib.StSolverOpts._fields_] == C_FIELDS
    o = stlib.st_default_opts()
    assert (o.nu1, o.nu2, o.smooth_sweeps, o.inner_cycles, o.use_graphs, o.use_tma) == (1, 1, 3, 1, 1, 1)
    assert o.recompute_slabs == 0
    assert (o.fuse_sweeps, o.fuse_start, o.fuse_restrict, o.fuse_update) == (1, 1, 1, 1)
    assert o.tol > 0 and o.krylov_rtol > 0
    S_FIELDS = [n.strip() for decl in re.findall(r"\b(?:int|double)\s+([^;]+);", _struct_text("st_stats_info"))
                for n in decl.split(",")]
    assert [f for f, _ in stlib.StStatsInfo._fields_] == S_FIELDS


def _struct_text(name):
    with open(os.path.join(ROOT, "include", "st.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    end = re.search(r"\}\s*" + name + r"\s*;", text)
    assert end, name
    start = text.rfind("typedef struct", 0, end.start())
    return text[text.index("{", start) + 1:end.start()]


@pytest.mark.parametrize("M", [1, 2, 3, 4, 5])
def test_host_collocation_setup_matches_oracle(stlib, M):
    tau, Q, lam, V, Vi = stlib.st_collocation(M)
    t0 = col.radau_right_nodes(M)
    Q0 = col.collocation_matrix(t0)
    l0, _ = col.q_eig(Q0)
    assert np.abs(tau - t0).max() < 1e-15
    assert np.abs(Q - Q0).max() < 1e-15
    assert np.abs(lam - l0).max() < 1e-14
    assert np.abs(Q @ V - V @ np.diag(lam)).max() < 1e-14
    assert np.abs(V @ Vi - np.eye(M)).max() < 1e-13
    # conjugate pairs are exact conjugates (the real transform relies on it)
    for p in range(M):
        if lam[p].imag > 0:
            assert lam[p + 1] == np.conj(lam[p])
            assert np.array_equal(V[:, p + 1], np.conj(V[:, p]))
    Pt, Rt = stlib.st_time_transfer(M)
    assert np.abs(Pt - col.time_prolongation(t0)).max() < 1e-13
    assert np.abs(Rt - col.time_restriction(t0)).max() < 1e-12


def test_plan_auto_mu_rule(stlib):
    """AUTO_MU bisects space while mu_l = nu dt/h^2 >= mu_crit, else the slabs
    (the mu rule of Section 4.2); SPACE bisects space only (SMG)."""
    p = stlib.make_problem((256, 256), stlib.PERIODIC, 1e-2, 256, 3, reaction=stlib.LOGISTIC, rho=1.0)
    info = stlib.st_plan(p)
    lv = [info.level[l] for l in range(info.levels)]
    assert lv[0].n[0] == 256 and lv[0].Nt == 256 and abs(lv[0].mu - 2.56) < 1e-12
    for a, b in zip(lv, lv[1:]):
        if a.next_kind == 1:
            assert a.mu >= 1.0 or a.Nt <= 4
            assert b.n[0] * 2 == a.n[0] and b.Nt == a.Nt and abs(b.dt - a.dt) < 1e-15
        else:
            assert a.next_kind == 2 and a.mu < 1.0
            assert b.n[0] == a.n[0] and 2 * b.Nt == a.Nt and abs(b.dt - 2 * a.dt) < 1e-15
    assert lv[-1].next_kind == 0 and lv[-1].Ns * 3 <= 96
    o = stlib.make_opts(coarsening=stlib.COARSEN_SPACE)
    info = stlib.st_plan(p, o)
    assert all(info.level[l].Nt == 256 for l in range(info.levels))
    assert info.level[info.levels - 1].Ns <= 16


def test_plan_space_nodes_rule(stlib):
    """SPACE_NODES (SMMG of Section 5.2) bisects space on every level and drops
    one collocation node per level until M = 1: M_l = max(M - l + 1, 1)."""
    p = stlib.make_problem((1025,), stlib.NEUMANN, 1.0, 8, 5)
    info = stlib.st_plan(p, stlib.make_opts(coarsening=stlib.COARSEN_SPACE_NODES, max_levels=7))
    lv = [info.level[l] for l in range(info.levels)]
    assert [l.M for l in lv] == [max(5 - l, 1) for l in range(len(lv))]
    assert [l.n[0] for l in lv] == [1025, 513, 257, 129, 65, 33, 17]
    assert all(l.Nt == 8 for l in lv)
    assert [l.next_kind for l in lv] == [3, 3, 3, 3, 1, 1, 0]


def test_plan_space_time_rule(stlib):
    """SPACE_TIME (the paper's STMG): space and slab bisection on one level
    while both are possible, then the direction that is left."""
    p = stlib.make_problem((64, 64), stlib.PERIODIC, 1.0, 16, 3)
    info = stlib.st_plan(p, stlib.make_opts(coarsening=stlib.COARSEN_SPACE_TIME))
    kinds = [info.level[l].next_kind for l in range(info.levels)]
    sizes = [(info.level[l].n[0], info.level[l].Nt) for l in range(info.levels)]
    assert kinds == [4, 4, 1, 1, 0], kinds
    assert sizes == [(64, 16), (32, 8), (16, 4), (8, 4), (4, 4)], sizes
    assert all(info.level[l].M == 3 for l in range(info.levels))
    assert info.level[1].dt == 2 * info.level[0].dt


def test_plan_space_time_respects_the_reaction_guard(stlib):
    """With a fast reaction the slabs are not bisected (2 dt |rho| max|lambda(Q)|
    above 1/2 would leave the coarse slab systems without meaning): SPACE_TIME
    then coarsens in space only, and slab bisection resumes where dt allows."""
    fast = stlib.make_problem((64, 64), stlib.PERIODIC, 1.0, 16, 3, T=1.0, reaction=stlib.LOGISTIC, rho=50.0)
    info = stlib.st_plan(fast, stlib.make_opts(coarsening=stlib.COARSEN_SPACE_TIME))
    kinds = [info.level[l].next_kind for l in range(info.levels)]
    assert 2 not in kinds and 4 not in kinds and kinds[0] == 1, kinds
    mild = stlib.make_problem((64, 64), stlib.PERIODIC, 1.0, 16, 3, T=1.0, reaction=stlib.LOGISTIC, rho=0.1)
    info = stlib.st_plan(mild, stlib.make_opts(coarsening=stlib.COARSEN_SPACE_TIME))
    assert info.level[0].next_kind == 4


def test_plan_dirichlet_and_neumann_sizes(stlib):
    p = stlib.make_problem((63,), stlib.DIRICHLET, 1.0, 16, 2)
    info = stlib.st_plan(p, stlib.make_opts(coarsening=stlib.COARSEN_SPACE))
    ns = [info.level[l].n[0] for l in range(info.levels)]
    assert ns == [63, 31, 15]  # stops at <= coarse_max_points (16)
    info = stlib.st_plan(p, stlib.make_opts(coarsening=stlib.COARSEN_SPACE, coarse_max_points=1))
    ns = [info.level[l].n[0] for l in range(info.levels)]
    assert ns == [63, 31, 15, 7, 3, 1]
    p = stlib.make_problem((65,), stlib.NEUMANN, 1.0, 8, 3)
    info = stlib.st_plan(p, stlib.make_opts(coarsening=stlib.COARSEN_SPACE, coarse_max_points=2))
    ns = [info.level[l].n[0] for l in range(info.levels)]
    assert ns == [65, 33, 17, 9, 5, 3, 2]
    h = [info.level[l].h[0] for l in range(info.levels)]
    assert all(abs(h[i + 1] - 2 * h[i]) < 1e-14 for i in range(len(h) - 1))


def test_invalid_arguments_rejected(stlib):
    for kw in [dict(nu=0.0), dict(M=6), dict(Nt=0)]:
        args = dict(shape=(16,), bc=stlib.PERIODIC, nu=1.0, Nt=4, M=2)
        args.update(kw)
        p = stlib.make_problem(args["shape"], args["bc"], args["nu"], args["Nt"], args["M"])
        with pytest.raises(stlib.StError) as ei:
            stlib.st_plan(p)
        assert ei.value.status == stlib.ST_ERR_INVALID_ARG


@pytest.mark.parametrize("Mf,Mc", [(2, 1), (3, 2), (5, 4), (5, 1), (4, 2)])
def test_host_node_transfer_matches_oracle(Mf, Mc):
    from paper_2006_12883_gb300 import stlib
    P, R = stlib.st_node_transfer(Mf, Mc)
    tf, tc = col.radau_right_nodes(Mf), col.radau_right_nodes(Mc)
    assert np.abs(P - col.node_prolongation(tf, tc)).max() < 1e-13
    assert np.abs(R - col.node_restriction(tf, tc)).max() < 1e-12
