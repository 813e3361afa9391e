"""GPU learned correction (training and inference kernels) against the oracle.

The library multiplies with BF16 copies of the weights and keeps biases,
activations and accumulation in FP32, so parity is checked against the FP64
oracle evaluated at the same BF16-rounded weights (FP32 rounding only:
1e-5 on outputs, 1e-4 on gradients), and the size of the BF16 effect itself
against the unrounded weights is stated (2e-2).  Training must lower the
loss, and the corrected flexible GMRES must still reach the oracle's field
with its true residual as the judge.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import discretization as D
from oracle import learned as NL
from oracle import solver as S

pytestmark = pytest.mark.gpu

CASE = W.small_case(40, 60, 8, 3, medium="grf", seed=21)


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _effective(theta32: np.ndarray) -> np.ndarray:
    """Weights as the library uses them: W in BF16, biases in FP32."""
    eff = theta32.astype(np.float64).copy()
    off = 0
    for name, shp in NL.shapes():
        n = int(np.prod(shp))
        if name.startswith("W"):
            eff[off:off + n] = torch.from_numpy(theta32[off:off + n]).to(torch.bfloat16).double().numpy()
        off += n
    return eff


@pytest.fixture(scope="module")
def setup():
    from paper_1410_5910_gb300 import PT_FP64, PolarTrace

    c = CASE.c_ext()
    om = CASE.omega(c)
    prob = D.make_problem(c, CASE.npml, CASE.h, om)
    solver = PolarTrace(CASE.nx, CASE.nz, CASE.npml, CASE.L, CASE.h, om, torch.from_numpy(c).cuda(), pml_C=prob.C,
                        precision=PT_FP64, max_sources=16, max_krylov=40, learned=True)
    return prob, solver


def _theta(seed, scale=0.05):
    g = np.random.default_rng(seed)
    th = (scale * g.standard_normal(NL.nparams())).astype(np.float32)
    return th


def test_forward_matches_oracle(setup):
    prob, solver = setup
    th = _theta(1)
    solver.set_correction(th)
    assert np.array_equal(solver.get_correction().numpy(), th)
    nseq = 5
    g = np.random.default_rng(2)
    X = g.standard_normal((nseq, NL.CIN, prob.nt))
    xg = torch.from_numpy(X.transpose(1, 0, 2).reshape(NL.CIN, -1).astype(np.float32)).cuda()
    y = solver.correction_forward(xg).cpu().numpy().reshape(NL.CIN, nseq, prob.nt).transpose(1, 0, 2)
    ref, _ = NL.forward(_effective(th), X.astype(np.float32).astype(np.float64))
    assert _rel(y, ref) < 1e-5
    ref32, _ = NL.forward(th.astype(np.float64), X)
    assert _rel(y, ref32) < 2e-2  # the BF16 weights themselves


def test_gradient_matches_oracle(setup):
    prob, solver = setup
    th = _theta(3, scale=0.08)
    solver.set_correction(th)
    nseq = 4
    g = np.random.default_rng(4)
    X = g.standard_normal((nseq, NL.CIN, prob.nt)).astype(np.float32)
    T = g.standard_normal((nseq, NL.CIN, prob.nt)).astype(np.float32)
    flat = lambda a: torch.from_numpy(a.transpose(1, 0, 2).reshape(NL.CIN, -1).copy()).cuda()  # noqa: E731
    loss, grad = solver.correction_grad(flat(X), flat(T))
    ref_loss, ref_grad = NL.loss_and_grad(_effective(th), X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    gg = grad.cpu().numpy().astype(np.float64)
    off = 0
    for name, shp in NL.shapes():
        n = int(np.prod(shp))
        assert _rel(gg[off:off + n], ref_grad[off:off + n]) < 1e-4, name
        off += n


def test_apply_correction_matches_oracle(setup):
    prob, solver = setup
    th = _theta(5)
    solver.set_correction(th)
    g = np.random.default_rng(6)
    v = g.standard_normal((3, solver.T4, prob.nt)) + 1j * g.standard_normal((3, solver.T4, prob.nt))
    v[1] *= 1e-3  # the RMS normalisation makes the map positively homogeneous
    z = solver.apply_correction(torch.from_numpy(v).cuda()).cpu().numpy()
    eff = _effective(th)
    for s in range(3):
        assert _rel(z[s], NL.correction_permuted(eff, v[s], CASE.L)) < 1e-5


def _pairs(solver, seeds, count):
    from paper_1410_5910_gb300.learned import solver_pairs

    rs, es = [], []
    for sd in seeds:
        g = np.random.default_rng(sd)
        pos = [(int(g.integers(1, CASE.nx + 1)), int(g.integers(1, CASE.nz // 3))) for _ in range(count)]
        f = torch.from_numpy(W.point_sources(CASE.nt, CASE.Nz, CASE.npml, CASE.h, pos)).cuda()
        r, e = solver_pairs(solver, f)
        rs.append(r)
        es.append(e)
    return torch.cat(rs), torch.cat(es)


def test_training_lowers_loss_and_corrected_gmres_reaches_oracle(setup):
    from paper_1410_5910_gb300 import PT_OPT_LEARNED
    from paper_1410_5910_gb300.learned import gate

    prob, solver = setup
    solver.set_option(PT_OPT_LEARNED, 0)
    g = np.random.default_rng(7)
    th = np.zeros(NL.nparams(), dtype=np.float32)
    off = 0
    for name, shp in NL.shapes():
        n = int(np.prod(shp))
        if name in ("W1", "W2", "W3"):
            fan = int(np.prod(shp[1:]))
            th[off:off + n] = g.uniform(-1, 1, n) * np.sqrt(3.0 / fan)
        off += n
    solver.set_correction(th)
    r, e = _pairs(solver, (11, 12, 13), 8)
    l0, l1 = solver.train_correction(r, e, steps=300, batch=4, lr=1e-3, seed=1)
    assert l1 < l0
    # held-out sources: the corrected flexible GMRES still reaches the oracle's
    # field, judged by its FP64 true residual
    g = np.random.default_rng(99)
    pos = [(int(g.integers(1, CASE.nx + 1)), int(g.integers(1, CASE.nz // 3))) for _ in range(6)]
    f = W.point_sources(CASE.nt, CASE.Nz, CASE.npml, CASE.h, pos)
    ft = torch.from_numpy(f).cuda()
    solver.set_option(PT_OPT_LEARNED, 1)
    u1, _, its1, rel1 = solver.solve(ft, tol=1e-10)
    mask = D.physical_mask(prob, CASE.nx, CASE.nz)
    for s in range(len(pos)):
        assert rel1[s] <= 1e-10
        ref = S.global_solve(prob, f[s])
        assert _rel(u1.cpu().numpy()[s][mask], ref[mask]) < 1e-8
    # the gain is measured, not assumed: the gate keeps the correction only if it
    # cut the iterations on validation sources, and the chosen form never needs
    # more iterations than the plain method there
    its_plain, its_corr, kept = gate(solver, ft, tol=1e-10)
    assert kept == (sum(its_corr) < sum(its_plain))
    _, _, its_chosen, rel_c = solver.solve(ft, tol=1e-10)
    assert sum(its_chosen) <= sum(its_plain) and max(rel_c) <= 1e-10
    solver.set_option(PT_OPT_LEARNED, 0)
    print(f"\nlearned correction: loss {l0:.3e} -> {l1:.3e}; iterations plain {its_plain} corrected {its_corr};"
          f" kept: {kept}")
