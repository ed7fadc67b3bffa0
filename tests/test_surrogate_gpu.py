"""The surrogate's tensor-core kernels against the FP64 network oracle.

The GEMM is checked element by element against the exact product of the
same BF16 operands, within the FP32 accumulation bound.  Gradients of a
forward and backward pass are checked against the oracle's backward pass
with BF16 rounding at the same points; training, prediction and the gate
are checked on a smooth synthetic response.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1702_04487_gb300 import surrogate
    return surrogate


@pytest.mark.parametrize("M_,N,K,lda,ldb", [
    (128, 256, 64, 64, 64), (1, 16, 8, 8, 8), (200, 16, 16, 16, 16), (300, 100, 136, 136, 144),
    (4096, 256, 256, 256, 256), (16, 256, 512, 512, 512), (129, 33, 40, 48, 40),
    (1000, 7, 72, 72, 72)])
def test_gemm_matches_exact_product(S, M_, N, K, lda, ldb):
    import torch
    g = torch.Generator().manual_seed(M_ * 7 + N)
    A = torch.randn(M_, lda, generator=g).to(torch.bfloat16)
    B = torch.randn(N, ldb, generator=g).to(torch.bfloat16)
    Ad, Bd = A.cuda(), B.cuda()
    Cd = torch.full((M_, N), float("nan"), device="cuda")
    S.gemm_bf16(Ad, Bd, M_, N, K, Cd, lda, ldb, N)
    a = A[:, :K].double().numpy()
    b = B[:, :K].double().numpy()
    ref = M.gemm_tn(a, b)
    bound = 4 * K * 2.0 ** -24 * (np.abs(a) @ np.abs(b).T) + 1e-30
    err = np.abs(Cd.cpu().double().numpy() - ref)
    assert (err <= bound).all(), float((err / bound).max())


def _data(n, seed):
    from paper_1702_04487_gb300 import surrogate as S
    rng = np.random.default_rng(seed)
    x = S.sample_inputs(n, seed)
    sd = x.std(0)
    z = (x - x.mean(0)) / np.where(sd > 0, sd, 1.0)  # the idle time is constant
    y = np.stack([3000 * np.exp(0.2 * z[:, 1] - 0.1 * z[:, 2] + 0.05 * z[:, 0] * z[:, 3]),
                  0.05 + 0.01 * np.tanh(z[:, 2] - 0.5 * z[:, 1]) + 0.002 * z[:, 6],
                  400 * np.exp(0.3 * z[:, 6] + 0.1 * z[:, 4]),
                  np.round(1 + np.clip(z[:, 5], -1, 1)) + 0.1 * rng.standard_normal(n)], 1)
    return x, y


def _oracle_view(sg, x, y):
    """Transformed inputs and targets, in the library's FP32 arithmetic."""
    im, isc, om, osc = sg.transform()
    cfg = sg.config
    xv = x.astype(np.float32).copy()
    for d in range(7):
        if (cfg["log_inputs"] >> d) & 1:
            xv[:, d] = np.log(xv[:, d])
    xt = ((xv - im) / isc).astype(np.float32)
    yv = y.astype(np.float32).copy()
    for d in range(4):
        if (cfg["log_outputs"] >> d) & 1:
            yv[:, d] = np.log(yv[:, d])
    yt = ((yv - om) / osc).astype(np.float32)
    return xt.astype(np.float64), yt.astype(np.float64)


def test_gradients_match_oracle(S):
    """The GPU's padded network (inputs 7 -> 16, outputs 4 -> 16) against
    the oracle's unpadded one: real entries match, padding gradients are 0."""
    H = 32
    sg = S.Surrogate(members=2, hidden=H, batch=64, seed=3)
    x, y = _data(256, 5)
    sg.set_data(x, y)
    xb, yb = x[:64], y[:64]
    g, loss = sg.gradients(xb, yb)
    xp, tp = _oracle_view(sg, xb, yb)
    w = np.array(sg.config["out_weight"])
    for mem in range(2):
        Wt, b = S.unpack(sg.get_params(mem).astype(np.float64), H)
        Wt[0], Wt[4], b[4] = Wt[0][:, :7], Wt[4][:4], b[4][:4]
        y_o, cache = M.forward(Wt, b, xp[:, :7], bf16=True)
        gW, gb = M.backward(Wt, b, cache, y_o, tp, weight=w, bf16=True)
        Wg, bg = S.unpack(g[mem].astype(np.float64), H)
        assert not Wg[0][:, 7:].any() and not Wg[4][4:].any() and not bg[4][4:].any()
        Wg[0], Wg[4], bg[4] = Wg[0][:, :7], Wg[4][:4], bg[4][:4]
        assert abs(loss[mem] - M.mse_loss(y_o, tp, weight=w)) < 1e-3 * loss[mem]
        for l in range(5):
            for got, ref in ((Wg[l], gW[l]), (bg[l], gb[l])):
                scale = np.abs(ref).max() + 1e-30
                assert np.abs(got - ref).max() < 2e-2 * scale, (mem, l, np.abs(got - ref).max() / scale)
                assert np.linalg.norm(got - ref) < 1e-2 * np.linalg.norm(ref) + 1e-30


def test_training_prediction_and_gate(S):
    sg = S.Surrogate(members=3, hidden=64, batch=128, seed=7, lr=2e-3)
    x, y = _data(2048, 11)
    sg.set_data(x[:1536], y[:1536])
    l0 = sg.train(1)
    l1 = sg.train(1500)
    assert np.isfinite(l1) and l1 < 0.1 * l0
    mean, sd, acc = sg.predict(x[1536:])
    err = np.abs(mean[:, 0] - y[1536:, 0]) / y[1536:, 0]
    assert np.median(err) < 0.05
    assert np.all(sd >= 0) and np.all(np.isfinite(mean))
    # gate: out of the input box is always rejected, the spread test follows tau
    far = x[1536:1552].copy()
    far[:, 0] = 179.0
    _, _, acc_far = sg.predict(far)
    assert not acc_far.any()
    # with the spread and distance tests off, exactly the queries inside the
    # training set's per-input box are accepted (the derived drive inputs of
    # held-out rows can fall outside it)
    sg.set_gate(1e9, 1e9, 1e9)
    _, _, acc_all = sg.predict(x[1536:])
    x32 = x.astype(np.float32)  # the box is kept and compared in FP32
    lo, hi = x32[:1536].min(0), x32[:1536].max(0)
    inside = np.all((x32[1536:] >= lo) & (x32[1536:] <= hi), axis=1)
    assert inside.mean() > 0.8
    assert np.array_equal(acc_all.astype(bool), inside)
    sg.set_gate(1e-9)
    _, _, acc_none = sg.predict(x[1536:])
    assert not acc_none.any()


def test_prediction_batch_sizes(S):
    """Any query count from 1 to beyond one tile gives the same rows."""
    sg = S.Surrogate(members=2, hidden=32, batch=32, seed=9)
    x, y = _data(300, 2)
    sg.set_data(x, y)
    full, _, _ = sg.predict(x, gate=False)
    for n in (1, 5, 127, 129, 300):
        part, _, _ = sg.predict(x[:n], gate=False)
        assert np.array_equal(part, full[:n])


@pytest.mark.slow
def test_surrogate_gain_over_the_lbm_alone(S):
    """Trained on 1024 lattice Boltzmann runs of the input box, the surrogate
    gated on the spread of its breakup time answers some held-out queries
    (about 10 % at this training size, 26 % with the bench's 4096 runs) near
    the LBM's breakup time and sends the rest to the LBM, taking no longer
    than the LBM alone.  (The droplet velocity just after pinch-off is
    not predictable to 1 % in this regime; its error is printed, not gated.)"""
    import time
    x_tr = S.sample_inputs(1024, 71)
    y_tr = S.lbm_outcomes(x_tr)
    ok = S.finite_rows(y_tr)
    assert ok.mean() > 0.9
    sg = S.Surrogate(members=5, hidden=256, batch=256, seed=5, lr=1e-3)
    sg.set_data(x_tr[ok], y_tr[ok])
    sg.train(6000)
    sg.set_gate(0.005, 1e9)
    x_ev = S.sample_inputs(128, 73)
    t0 = time.perf_counter()
    y_ev = S.lbm_outcomes(x_ev)
    t_lbm = time.perf_counter() - t0
    svc = S.SurrogateService(sg)
    sg.predict(x_ev[:16])
    t0 = time.perf_counter()
    y_sv, acc = svc.query(x_ev)
    t_svc = time.perf_counter() - t0
    fin = S.finite_rows(y_ev)
    sel = acc & fin
    err = S.relative_error(y_sv[sel, 0], y_ev[sel, 0])
    err_v = S.relative_error(y_sv[sel, 1], y_ev[sel, 1])
    print("gated surrogate: accepted %d/%d, breakup error p95 %.4f, velocity error p50 %.4f, "
          "%.2fx faster than the LBM" % (acc.sum(), len(x_ev), np.percentile(err, 95),
                                          np.median(err_v), t_lbm / t_svc))
    assert acc.mean() > 0.02
    # on this small training set and a dozen accepted queries: nearly all
    # within 1 %, none far off (the bench, with 4096 runs, holds >= 95 %)
    assert (err <= 0.01).mean() >= 0.9 and err.max() < 0.03
    # rejected queries carry the LBM's own answer
    rej = ~acc & fin
    assert np.allclose(y_sv[rej], y_ev[rej], rtol=1e-6)
    assert t_svc < 1.1 * t_lbm  # the fallback batch is a subset of the LBM's
