"""Per-kernel timing of instrumented runs (ufg_profile_enable / ufg_profile_read): the records
cover the solve's kernels with positive device time, the algorithmic bytes follow the operand
count of each launch, and the instrumented solve (its own graphs, with event nodes) returns the
same solution as the ordinary one."""
import pytest
import torch

from paper_1008_3647_gb300.inputs import field_and_source

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ufg():
    from paper_1008_3647_gb300 import ufg as u
    u.load()
    return u


def _probs(shapes):
    out = []
    for nx, nt, seed in shapes:
        sg, b = field_and_source(nx, nt, seed)
        out.append({"nx": nx, "ntau": nt, "sigma": torch.from_numpy(sg).cuda(),
                    "b": torch.from_numpy(b).cuda(),
                    "x": torch.zeros(nt, nx, nx, nx, dtype=torch.float64, device="cuda")})
    return out


def test_profile_records_batched_solve(ufg):
    shapes = [(8, 40, 1), (16, 48, 14)]  # 16^3 FP32 takes the fused M1 kernel
    ref = _probs(shapes)
    ufg.ufg_solve_batch(ref, "wce", {"order": 2}, tol=1e-10, precision=ufg.UFG_MIXED)
    probs = _probs(shapes)
    ufg.ufg_profile_enable(True)
    try:
        stats = ufg.ufg_solve_batch(probs, "wce", {"order": 2}, tol=1e-10,
                                    precision=ufg.UFG_MIXED)
    finally:
        ufg.ufg_profile_enable(False)
    assert all(s["status"] == ufg.UFG_OK for s in stats)
    for a, b in zip(ref, probs):  # same kernels in the same order: bit-identical solutions
        assert torch.equal(a["x"], b["x"])
    ks = ufg.ufg_profile_read()
    names = {k["name"] for k in ks}
    assert any(n.startswith("slice kin") for n in names), names
    assert any(n.startswith("recurrence") for n in names), names
    assert any(n.startswith("vec bi_x f32") for n in names), names
    assert "scalar" in names
    assert [k["total_ms"] for k in ks] == sorted((k["total_ms"] for k in ks), reverse=True)
    for k in ks:
        # classes whose launches found every problem stopped (e.g. restart-only steps) move
        # nothing; the kernels of the iteration body do
        assert k["launches"] > 0 and k["total_ms"] > 0 and k["bytes"] >= 0
        assert k["gbs"] < 20000  # far above any HBM or L2 rate would mean miscounted bytes
    for prefix in ("slice kin", "slice m1w", "recurrence acc1", "vec bi_x f32"):
        assert any(k["name"].startswith(prefix) and k["bytes"] > 0 for k in ks), prefix
    # a vec bi_x launch over all running problems moves 7 FP32 vectors per site
    bx = [k for k in ks if k["name"] == "vec bi_x f32"][0]
    sites = sum(nx ** 3 * nt for nx, nt, _ in shapes)
    assert bx["bytes"] <= bx["launches"] * 7 * 4 * sites
    # disabled: nothing more is recorded
    n0 = len(ufg.ufg_profile_read())
    ufg.ufg_solve_batch(_probs(shapes[:1]), "wce", {"order": 1}, tol=1e-8)
    assert sum(k["launches"] for k in ufg.ufg_profile_read()) == sum(k["launches"] for k in ks)
    assert len(ufg.ufg_profile_read()) == n0


def test_profile_single_problem_solve(ufg):
    nx, nt = 8, 24
    sg, b = field_and_source(nx, nt, 3)
    lat = ufg.Lattice(nx, nt)
    field = ufg.Field(lat, torch.from_numpy(sg).cuda())
    solver = ufg.Solver(lat)
    solver.ufg_set_preconditioner("cheb", degree=8)
    ufg.ufg_profile_enable(True)
    try:
        x, st = solver.ufg_solve_cg_normal(field, torch.from_numpy(b).cuda(), tol=1e-10)
    finally:
        ufg.ufg_profile_enable(False)
    assert st["status"] == ufg.UFG_OK
    ks = ufg.ufg_profile_read()
    slices = [k for k in ks if k["name"].startswith("slice kin")]
    assert slices and all(k["bytes"] > 0 for k in slices)


def test_profile_single_problem_wce_solve_in_momentum_basis(ufg):
    # a mixed BiCGStab + WCE2 solve of one 16^3 lattice (momentum basis, every flagged launch
    # inside the solver's captured graphs) runs and is recorded under the profiler
    nx, nt = 16, 64
    sg, b = field_and_source(nx, nt, 4)
    lat = ufg.Lattice(nx, nt)
    field = ufg.Field(lat, torch.from_numpy(sg).cuda())
    solver = ufg.Solver(lat)
    solver.ufg_set_preconditioner("wce", order=2, euler="euler23")
    bd = torch.from_numpy(b).cuda()
    _, st0 = solver.ufg_solve_bicgstab_two_step(field, bd, tol=1e-10, precision=ufg.UFG_MIXED)
    ufg.ufg_profile_enable(True)
    try:
        x, st = solver.ufg_solve_bicgstab_two_step(field, bd, tol=1e-10,
                                                   precision=ufg.UFG_MIXED)
    finally:
        ufg.ufg_profile_enable(False)
    assert st["status"] == ufg.UFG_OK, st
    assert st["iterations"] == st0["iterations"]
    ks = ufg.ufg_profile_read()
    names = {k["name"] for k in ks}
    assert any(n.startswith("recurrence") for n in names), names
    assert any(n.startswith("slice m1w") for n in names), names
    assert all(k["launches"] > 0 and k["total_ms"] > 0 for k in ks)
