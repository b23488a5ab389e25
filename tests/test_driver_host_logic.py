"""Host logic of the Sec. 3.8 loop on the CPU: the library's own loop
(afd_topology_run, the code afd_constrained_topology runs on a mesh) driven
by analyses the oracle answers, with the oracle's level-set cut.  The AL
scalars come from the library (Eqs. 3.11, 3.12, 3.18).  Checks steps 4 and
7-9 of Sec. 3.8 and the hard / soft split of Sec. 3.6 without a GPU."""
import numpy as np
import pytest

from oracle import buckling, fe, levelset, modal, sensitivity
from synthetic import axial_face_load, clamp_face_x0, edge_load


@pytest.fixture(scope="module")
def afd():
    from paper_2203_15115_gb300 import build

    build.build()
    import paper_2203_15115_gb300 as afd

    afd.lib()
    return afd


_MESHES = {}


class OracleMesh:
    """The subset of Mesh that the driver calls, computed by the oracle.  Like
    the library's level-set update, the cut writes the new moduli into the
    mesh (kept 1, the rest e_void)."""

    class _Opt:
        e_void = 1e-3

    def __init__(self, nx, ny, nz, f, fixed):
        self.nx, self.ny, self.nz, self.f, self.fixed = nx, ny, nz, f, fixed
        self.nelem = nx * ny * nz
        self.options = self._Opt()
        self.h = len(_MESHES) + 1
        _MESHES[self.h] = self
        self.E = None
        self.u = None
        self.calls = {"solve": 0, "modal": 0, "buckling": 0}

    def set_element_moduli(self, E):
        self.E = np.asarray(E, dtype=np.float64).copy()
        self.u = None

    def solve(self, tol, warm_start=False):
        self.calls["solve"] += 1
        self.u = fe.solve_direct(fe.assemble(self.nx, self.ny, self.nz, self.E), self.f, self.fixed)
        return [{"iters": 1, "rel_residual": 0.0}]

    def compliance(self):
        assert self.u is not None, "the static solution was discarded"
        return np.array([fe.compliance(self.f, self.u)])

    def pnorm_stress(self, p):
        return np.array([sensitivity.pnorm(sensitivity.element_von_mises(self.nx, self.ny, self.nz, self.E, self.u), p)])

    def sensitivity(self, kind, out):
        out[0] = sensitivity.strain_energy(self.nx, self.ny, self.nz, self.E, self.u)

    def stress_sensitivity(self, p, tol, out):
        # Eq. 3.3 with its adjoint: K lambda = -d sigma_PN / d u on the free DOFs
        assert self.u is not None, "the stress field needs the static solution"
        g = sensitivity.pnorm_stress_gradient(self.nx, self.ny, self.nz, self.E, self.u, p)
        lam = fe.solve_direct(fe.assemble(self.nx, self.ny, self.nz, self.E), -g, self.fixed)
        out[0] = sensitivity.stress_topological_sensitivity(self.nx, self.ny, self.nz, self.E, self.u, lam)

    def modal(self, n, rho=1.0, tol=1e-6):
        self.calls["modal"] += 1
        lam, phi = modal.modes(self.nx, self.ny, self.nz, self.E, self.fixed, n, rho=rho)
        self._modes = (lam, phi, rho)
        self.u = None
        return lam, {"steps": 1}

    def eigen_sensitivity(self, out):
        lam, phi, rho = self._modes
        out[0] = modal.eigen_sensitivity(self.nx, self.ny, self.nz, self.E, phi[0], lam[0], rho)

    def buckling(self, n, tol=1e-6):
        assert self.u is not None, "buckling needs the static state"
        self.calls["buckling"] += 1
        lam, phi, S = buckling.buckling(self.nx, self.ny, self.nz, self.E, self.f, self.fixed, n)
        self._buck = (lam, phi, S)
        self.u = None
        return lam, {"steps": 1}

    def buckling_sensitivity(self, out):
        lam, phi, S = self._buck
        out[0] = buckling.buckling_sensitivity(self.nx, self.ny, self.nz, self.E, S, phi[0], lam[0])


def run_oracle_topology(afd, m, E0, compliance=None, stress=None, eigen=None, buckling=None, soft=(), p=8.0,
                        dv0=0.05, v_min=0.05, max_fea=200, casting=None, on_design=None, rho=1.0, eig_tol=1e-6,
                        tol=1e-6):
    """afd_topology_run with the oracle mesh's analyses and the oracle's cut
    (combination of Eq. 3.17, casting scan, top-k of Eq. 3.6, new moduli)."""
    sp = afd.topology_spec(compliance, stress, eigen, buckling, soft, p, dv0, None, v_min, 0.01, max_fea, tol,
                           eig_tol, rho, casting)
    act = [sp.bound[c] > 0 for c in range(4)]
    ne = m.nelem
    fields, state, feas = {}, {"kept": np.ones(ne, np.uint8)}, {}
    m.set_element_moduli(np.asarray(E0, dtype=np.float64))

    def field(fn):
        f = np.zeros((1, ne), np.float32)
        fn(f)
        return f[0]

    def analyse(warm):
        m.solve(tol, warm_start=warm)
        vals = [float(m.compliance()[0]), None, None, None]
        if act[0]:
            fields[0] = field(lambda f: m.sensitivity(0, f))
        if act[1]:
            vals[1] = float(m.pnorm_stress(p)[0])
            fields[1] = field(lambda f: m.stress_sensitivity(p, tol, f))
        if act[3]:
            lam, _ = m.buckling(1, tol=eig_tol)
            vals[3] = float(lam[0])
            fields[3] = field(m.buckling_sensitivity)
        if act[2]:
            lam, _ = m.modal(1, rho=rho, tol=eig_tol)
            vals[2] = float(lam[0])
            fields[2] = field(m.eigen_sensitivity)
        return vals, 1, 0.0

    def save():
        feas["E"], feas["kept"] = m.E.copy(), state["kept"].copy()

    def restore():
        m.set_element_moduli(feas["E"])
        state["kept"] = feas["kept"].copy()

    def cut(w, v):
        idx = [c for c in range(4) if act[c]]
        T = levelset.combine(np.stack([fields[c] for c in idx]).astype(np.float32),
                             np.asarray([w[c] for c in idx], dtype=np.float64))
        if casting is not None:
            T = levelset.casting_scan(T, m.nx, m.ny, m.nz, *casting)
        sel, _ = levelset.select_top(T, levelset.keep_count(v, T.size))
        state["kept"] = sel.astype(np.uint8)
        m.set_element_moduli(levelset.apply_topology(sel, m.options.e_void))
        if on_design:
            on_design(m.E.copy())

    res = afd.afd_topology_run(sp, analyse, save, restore, cut)
    res["kept"], res["E"] = feas["kept"], feas["E"]
    return res


def _check_steps(hist, conv=0.01):
    """Steps 4 and 7-9 of Sec. 3.8 on the records: after a violated hard
    constraint the step halves and the next design is the last feasible one
    minus the new step; the target drops only when the previous analysis was
    feasible too and J moved by at most `conv` since it."""
    feasible_v = 1.0
    for i in range(len(hist) - 1):
        a, b = hist[i], hist[i + 1]
        assert b["v"] == b["target"]
        if a["violated"]:
            assert b["dv"] == a["dv"] / 2
            assert b["v"] == pytest.approx(feasible_v - b["dv"], abs=1e-12)
        else:
            feasible_v = a["v"]
            if b["target"] < a["target"]:
                assert i > 0 and not hist[i - 1]["violated"]
                assert abs(a["J"] - hist[i - 1]["J"]) <= conv * abs(hist[i - 1]["J"])
                assert b["target"] == pytest.approx(a["target"] - a["dv"], abs=1e-12)
            else:
                assert b["target"] == a["target"]


def _replay_al(hist, name):
    mu, gamma, g_prev = levelset.MU0, levelset.GAMMA0, 0.0
    for k, h in enumerate(hist, start=1):
        g = h["g"][name]
        mu = levelset.multiplier_update(mu, gamma, g)
        gamma = levelset.penalty_update(gamma, g, g_prev, k)
        g_prev = g
        assert h["mu"][name] == pytest.approx(mu, rel=1e-12, abs=1e-12)
        assert h["gamma"][name] == pytest.approx(gamma, rel=1e-12)


def test_hard_compliance_and_eigenvalue_steps(afd):
    nx, ny, nz = 10, 4, 3
    f, fixed = edge_load(nx, ny, nz), clamp_face_x0(nx, ny, nz)
    m = OracleMesh(nx, ny, nz, f, fixed)
    res = run_oracle_topology(afd, m, np.ones(nx * ny * nz), compliance=1.6, eigen=0.9, dv0=0.1, v_min=0.3,
                              max_fea=25)
    hist = res["history"]
    assert res["stop"] in ("dv_min", "v_min", "max_fea")
    for h in hist:
        assert h["violated"] == (h["g"]["J"] > 0 or h["g"]["lambda"] > 0)
    _replay_al(hist, "J")
    _replay_al(hist, "lambda")
    assert any(h["violated"] for h in hist) and any(b["target"] < a["target"] for a, b in zip(hist, hist[1:]))
    _check_steps(hist)
    # the final design is feasible for both hard constraints under the oracle
    E = res["E"]
    J0 = res["reference"]["J"]
    lam0 = res["reference"]["lambda"]
    u = fe.solve_direct(fe.assemble(nx, ny, nz, E), f, fixed)
    assert fe.compliance(f, u) <= 1.6 * J0 * (1 + 1e-12)
    assert modal.modes(nx, ny, nz, E, fixed, 1)[0][0] >= 0.9 * lam0 * (1 - 1e-9)
    assert int(res["kept"].sum()) == levelset.keep_count(res["volume_fraction"], E.size)
    # the modal analysis discards the static solution: the static fields come first, every analysis
    assert m.calls["modal"] == m.calls["solve"] == res["fea"]


def test_soft_buckling_never_rejects_and_unconverged_targets_stay(afd):
    nx, ny, nz = 10, 3, 2
    f, fixed = axial_face_load(nx, ny, nz, -1.0), clamp_face_x0(nx, ny, nz)
    m = OracleMesh(nx, ny, nz, f, fixed)
    res = run_oracle_topology(afd, m, np.ones(nx * ny * nz), compliance=1.5, buckling=2.0, soft=("P",),
                              dv0=0.1, v_min=0.4, max_fea=12)
    hist = res["history"]
    assert all(h["g"]["P"] > 0 for h in hist)          # P >= 2 P_0 is never met ...
    for h in hist:
        assert h["violated"] == (h["g"]["J"] > 0)       # ... and never counts
    _replay_al(hist, "P")
    assert m.calls["buckling"] == res["fea"]
    assert any(h["violated"] for h in hist)
    _check_steps(hist)
    with pytest.raises(ValueError):
        afd.run_constrained_topology(m, np.ones(nx * ny * nz), compliance=1.5, soft=("J",))


def test_hard_compliance_and_stress_steps(afd):
    """Both constraints of the paper's static problem hard: J <= 1.5 J_0 and
    sigma_PN(p = 8) <= 1.3 sigma_0.  Every record's violation flag follows the
    two g values, both multipliers follow Eqs. 3.11-3.12, steps 4 and 7-9 hold,
    and the final design meets both constraints under the oracle."""
    nx, ny, nz = 12, 4, 3
    f, fixed = edge_load(nx, ny, nz), clamp_face_x0(nx, ny, nz)
    m = OracleMesh(nx, ny, nz, f, fixed)
    res = run_oracle_topology(afd, m, np.ones(nx * ny * nz), compliance=1.5, stress=1.3, p=8.0, dv0=0.1,
                              v_min=0.3, max_fea=25)
    hist = res["history"]
    for h in hist:
        assert h["violated"] == (h["g"]["J"] > 0 or h["g"]["sigma"] > 0)
    _replay_al(hist, "J")
    _replay_al(hist, "sigma")
    _check_steps(hist)
    assert any(h["violated"] for h in hist)
    E = res["E"]
    u = fe.solve_direct(fe.assemble(nx, ny, nz, E), f, fixed)
    assert fe.compliance(f, u) <= 1.5 * res["reference"]["J"] * (1 + 1e-12)
    vm = sensitivity.element_von_mises(nx, ny, nz, E, u)
    assert sensitivity.pnorm(vm, 8.0) <= 1.3 * res["reference"]["sigma"] * (1 + 1e-12)


@pytest.mark.parametrize("axis,parting", [(2, 0), (1, 2)])
def test_casting_designs_have_no_undercut(afd, axis, parting):
    """Sec. 3.7 inside the Sec. 3.8 loop: with a casting direction every design
    the driver cuts, and the final feasible one, keeps on each line along the
    axis and on each side of the parting plane a run of elements that starts
    at the plane (the part can be drawn from its mould)."""
    nx, ny, nz = 10, 4, 4
    f, fixed = edge_load(nx, ny, nz), clamp_face_x0(nx, ny, nz)
    m = OracleMesh(nx, ny, nz, f, fixed)
    designs = []
    res = run_oracle_topology(afd, m, np.ones(nx * ny * nz), compliance=2.0, dv0=0.1, v_min=0.4, max_fea=12,
                              casting=(axis, parting), on_design=designs.append)
    designs.append(res["E"])
    _check_steps(res["history"])
    for E in designs:
        a = np.moveaxis((E == 1.0).reshape(nz, ny, nx), {0: 2, 1: 1, 2: 0}[axis], 0)
        n = a.shape[0]
        for half in (a[parting:], a[:parting][::-1]):       # each half ordered away from the plane
            if half.shape[0] == 0:
                continue
            run = np.cumprod(half, axis=0)                   # kept and every element before it kept
            assert np.array_equal(run, half), "undercut"
    assert any(not np.all(E == 1.0) for E in designs)


def test_topology_loop_refuses_bad_specs_and_stops_on_callback_errors(afd):
    """The library checks the spec before any analysis, and an error in a
    callback ends the run with that error (here a Python exception, re-raised)."""
    calls = []

    def analyse(warm):
        calls.append(warm)
        return [1.0, None, None, None], 1, 0.0

    noop = lambda *a: None
    sp = afd.topology_spec(compliance=1.5, soft=("J",))
    with pytest.raises(afd.AFDError) as e:
        afd.afd_topology_run(sp, analyse, noop, noop, noop)
    assert e.value.code == afd.AFD_ERR_INVALID_ARG and not calls
    with pytest.raises(afd.AFDError):
        afd.afd_topology_run(afd.topology_spec(), analyse, noop, noop, noop)
    assert not calls

    def bad_cut(w, v):
        raise RuntimeError("cut failed")

    with pytest.raises(RuntimeError, match="cut failed"):
        afd.afd_topology_run(afd.topology_spec(compliance=1.5, dv0=0.1), analyse, noop, noop, bad_cut)
    # first analysis, J unchanged -> feasible, cut raised: no further analysis
    assert calls == [False]


def test_topology_loop_follows_the_steps_on_scripted_values(afd):
    """Scripted compliance values (no mesh): feasible, feasible and settled ->
    the target drops; violated -> back to the feasible design with half the
    step; the records carry the state before each decision."""
    J = iter([1.0, 1.2, 1.205, 2.0, 1.3, 1.31, 1.311, 1.312])
    log = []

    def analyse(warm):
        return [next(J), None, None, None], 3, 1e-7

    res = afd.afd_topology_run(afd.topology_spec(compliance=1.5, dv0=0.1, v_min=0.5, max_fea=7),
                               analyse, lambda: log.append("save"), lambda: log.append("restore"),
                               lambda w, v: log.append(("cut", round(v, 12))))
    h = res["history"]
    # the re-analysis of the restored design feeds the next cut and is not recorded on its own (fea 5)
    assert [r["fea"] for r in h] == [1, 2, 3, 4, 6, 7] and res["stop"] == "max_fea" and res["fea"] == 7
    assert [round(r["target"], 12) for r in h] == [0.9, 0.9, 0.9, 0.8, 0.85, 0.85]
    assert [r["violated"] for r in h] == [False, False, False, True, False, False]
    assert h[4]["dv"] == 0.05 and h[4]["v"] == 0.85 and h[3]["dv"] == 0.1
    assert log == ["save", "save", ("cut", 0.9), "save", ("cut", 0.9), "save", ("cut", 0.8), "restore",
                   ("cut", 0.85), "save", ("cut", 0.85)]
    assert res["volume_fraction"] == 0.85
