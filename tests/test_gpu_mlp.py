"""Warm-start encoder: gradients, forward pass and Adam against the FP64 oracle
(oracle/mlp.py), and what the trained network gains over starting the per-cell
projection from zero.

Tolerances: FP32 GEMM sums of <= 3000 products (relative error ~1e-6) and FP32
erf-based gelu: loss within 1e-5, forward outputs and gradients within 1e-4
(max-norm relative per tensor), one Adam step within 1e-5.
"""
import numpy as np
import pytest

import synth
from tests.test_gpu_parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gmf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_20509_gb300 as g
    return g


def f32(P):
    return {k: np.asarray(v, dtype=np.float32).astype(np.float64) for k, v in P.items()}


def bf16(a):
    """Round to BF16 (nearest even) through FP32, as the tensor-core layer rounds its operands."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("dims,rows,y16", [((3000, 256, 256, 20), 300, True), ((200, 64, 32, 5), 130, False),
                                           ((64, 16, 16, 3), 1, True)])
def test_mixed_first_layer_matches_oracle_on_bf16_operands(gmf, dims, rows, y16):
    """The tensor-core first layer rounds W1 and log(1 + y) to BF16 and accumulates
    in FP32: against the FP64 oracle fed the same rounded operands only the
    accumulation order differs (~1e-6 relative), so the outputs agree within
    1e-4 (max-norm relative), with ragged rows (300, 130, 1 = not multiples of
    128) and a K tail (200 = 3 x 64 + 8)."""
    from oracle import mlp
    rng = np.random.default_rng(40)
    P = f32(mlp.init_params(*dims, seed=8))
    for k in ("b1", "b2", "b3"):
        P[k] = f32({k: 0.1 * rng.standard_normal(P[k].shape)})[k]
    Y = rng.poisson(rng.gamma(0.5, 4.0, size=(rows, dims[0])))
    Y[rng.random(Y.shape) < 0.02] += 400   # some counts beyond the 256-entry table
    Y = Y.astype(np.uint16 if y16 else np.int32)
    net = gmf.MLP(*dims, max_batch=max(rows, 128))
    net.set_params(P)
    net.set_precision("mixed")
    Yd = torch.from_numpy(Y.view(np.int16) if y16 else Y).cuda()
    out = net.forward(Yd).cpu().numpy()
    Pb = dict(P, W1=bf16(P["W1"]))
    ref, _ = mlp.forward_x(Pb, bf16(np.log1p(Y.astype(np.float64))))
    assert rel(out, ref) <= 1e-4, rel(out, ref)
    # and the FP32 path differs from it by the BF16 rounding, not more
    net.set_precision("fp32")
    out32 = net.forward(Yd).cpu().numpy()
    ref32, _ = mlp.forward(P, Y.astype(np.float64))
    assert rel(out32, ref32) <= 1e-4
    assert rel(out, ref32) <= 5e-2


def test_mixed_encoder_rejects_unsupported_shapes(gmf):
    net = gmf.MLP(100, 24, 16, 4, max_batch=64)
    with pytest.raises(gmf.GmfError):
        net.set_precision("mixed")          # n_h1 = 24 is not a multiple of 16
    net = gmf.MLP(10, 32, 16, 4, max_batch=64)
    net.set_precision("mixed")
    Y = torch.zeros((5, 10), dtype=torch.int32, device="cuda")
    with pytest.raises(gmf.GmfError):
        net.forward(Y)                      # 10 int32 counts per row: 40 bytes, not a multiple of 16


@pytest.mark.parametrize("dims,rows,y16", [((300, 40, 24, 5), 37, False), ((3000, 256, 256, 20), 256, True)])
def test_mlp_loss_and_gradients_match_oracle(gmf, dims, rows, y16):
    from oracle import mlp
    rng = np.random.default_rng(11)
    P = f32(mlp.init_params(*dims, seed=3))
    for k in ("b1", "b2", "b3"):
        P[k] = f32({k: 0.1 * rng.standard_normal(P[k].shape)})[k]
    Y = rng.poisson(2.0, size=(rows, dims[0])).astype(np.uint16 if y16 else np.int32)
    T = rng.standard_normal((rows, dims[3])).astype(np.float32)
    net = gmf.MLP(*dims, max_batch=rows)
    net.set_params(P)
    Yd = torch.from_numpy(Y.view(np.int16) if y16 else Y).cuda()   # uint16 counts travel as raw 16-bit words
    loss = net.loss_grad(Yd, torch.from_numpy(T).cuda())
    lref, gref = mlp.loss_grad(P, Y.astype(np.float64), T.astype(np.float64))
    assert float(loss.item()) == pytest.approx(lref, rel=1e-5)
    g = net.get_grads()
    for k in mlp.NAMES:
        assert rel(g[k], gref[k]) <= 1e-4, (k, rel(g[k], gref[k]))
    out = net.forward(Yd).cpu().numpy()
    oref, _ = mlp.forward(P, Y.astype(np.float64))
    assert rel(out, oref) <= 1e-4


def test_mlp_adam_step_matches_oracle(gmf):
    from oracle import mlp
    rng = np.random.default_rng(12)
    dims = (120, 32, 16, 4)
    P = f32(mlp.init_params(*dims, seed=5))
    Y = rng.poisson(3.0, size=(50, dims[0])).astype(np.int32)
    T = rng.standard_normal((50, dims[3])).astype(np.float32)
    net = gmf.MLP(*dims, max_batch=64)
    net.set_params(P)
    net.loss_grad(torch.from_numpy(Y).cuda(), torch.from_numpy(T).cuda())
    net.adam(1e-3)
    got = net.get_params()
    _, g = mlp.loss_grad(P, Y.astype(np.float64), T.astype(np.float64))
    mlp.adam_step(P, g, {}, lr=1e-3)
    for k in mlp.NAMES:
        assert rel(got[k], P[k]) <= 1e-5, k


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_mlp_training_is_deterministic_and_learns(gmf, precision):
    from oracle import mlp
    rng = np.random.default_rng(13)
    dims = (200, 64, 64, 6)
    W = rng.standard_normal((dims[3], dims[0])) * 0.1
    Y = rng.poisson(2.0, size=(900, dims[0])).astype(np.int32)
    T = (np.log1p(Y) @ W.T).astype(np.float32)
    P0 = f32(mlp.init_params(*dims, seed=1))
    runs = []
    for _ in range(2):
        net = gmf.MLP(*dims, max_batch=128)
        net.set_precision(precision)
        net.set_params(P0)
        losses = net.train(torch.from_numpy(Y).cuda(), torch.from_numpy(T).cuda(), epochs=15, batch=128, lr=3e-3,
                           seed=4)
        runs.append((losses, net.get_params()))
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    for k in mlp.NAMES:
        np.testing.assert_array_equal(runs[0][1][k], runs[1][1][k])
    assert runs[0][0][-1] < 0.5 * runs[0][0][0]


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_warm_start_beats_cold_start(gmf, precision):
    """Fit on training cells, orthogonalise (B1), train the encoder on (counts,
    scores), then project held-out cells by Fisher scoring from the network's
    scores and from zero. Fisher scoring minimises the penalised objective
    0.5 deviance + 0.5 lambda_U |u|^2 (lambda_Gamma = 0 here), so the gap to a
    40-step cold fit is measured on it: the warm start is much closer after one
    step and after three."""
    from oracle import mlp
    n_fit, n_new, m, d = 3000, 800, 480, 6
    prob = synth.make_problem(n_fit + n_new, m, 3, 1, d, "negbin", seed=17, zero_frac=0.7, offset=True)
    fit = slice(0, n_fit)
    new = slice(n_fit, n_fit + n_new)
    Yfit = np.ascontiguousarray(prob.Y[fit])
    sub = synth.Problem(Y=Yfit, X=prob.X[fit], Z=prob.Z, offset=prob.offset[fit], B=prob.B, Gamma=prob.Gamma[fit],
                        U=prob.U[fit], V=prob.V, nb_size=prob.nb_size, family="negbin")
    start = synth.crude_start(sub, d, seed=17)
    rp, cp = synth.partitions(n_fit, m, 17)
    settings = synth.fit_settings(k0=0.05, alpha_mode=1)
    model = gmf.Model(torch.from_numpy(Yfit).cuda(), sub.X, sub.Z, sub.offset, start, family="negbin", nb_row=500,
                      nb_col=160, row_perm=rp, col_perm=cp, settings=settings, precision="mixed")
    for s in synth.sweep_orders(n_fit, m, 500, 160, 40, 17):
        model.epoch(s)
    model.orthogonalize("B1")
    # Targets: the training cells' scores re-solved per cell given the fitted column side
    # (what the method produces for them with B, V and the shape fixed).
    Yfd = torch.from_numpy(Yfit).cuda()
    Ufit, _, _ = model.project_cells(Yfd, torch.from_numpy(sub.X).cuda(), torch.from_numpy(sub.offset).cuda(), None,
                                     n_steps=15, with_dev=False)
    net = gmf.MLP(m, 256, 256, d, max_batch=256)
    net.set_precision(precision)
    net.set_params(f32(mlp.init_params(m, 256, 256, d, seed=2)))
    losses = net.train(Yfd, Ufit, epochs=60, batch=256, lr=1e-3, seed=5)
    assert losses[-1] < 0.1 * losses[0]
    Ynew = torch.from_numpy(np.ascontiguousarray(prob.Y[new])).cuda()
    Xnew = torch.from_numpy(prob.X[new]).cuda()
    onew = torch.from_numpy(prob.offset[new]).cuda()
    Uwarm = net.forward(Ynew)
    lam_u = settings["lambda_"][2]

    def objective(U, G, D):
        return 0.5 * D.double() + 0.5 * lam_u * (U.double() ** 2).sum(1) + 0.5 * settings["lambda_"][1] * \
            (G.double() ** 2).sum(1)

    ref = objective(*model.project_cells(Ynew, Xnew, onew, None, n_steps=40))
    gaps = {}
    for steps in (1, 3):
        gaps[("warm", steps)] = float((objective(*model.project_cells(Ynew, Xnew, onew, Uwarm, n_steps=steps)) -
                                       ref).mean())
        gaps[("cold", steps)] = float((objective(*model.project_cells(Ynew, Xnew, onew, None, n_steps=steps)) -
                                       ref).mean())
    scale = float(ref.abs().mean())
    assert gaps[("warm", 1)] < 0.2 * gaps[("cold", 1)], gaps
    assert gaps[("warm", 3)] < 0.5 * gaps[("cold", 3)] + 1e-6 * scale, gaps
