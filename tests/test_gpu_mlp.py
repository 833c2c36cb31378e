"""GPU tests of the warm-start network (lbm_mlp_*) against the FP64 oracle (oracle/mlp.py).

Tolerances:
* tensor-core GEMM: products of bfloat16 values are exact in FP32 and the FP32 sum of K
  of them is within K 2^-24 sum|a b| of the exact sum; checked at 2 K 2^-24 sum|a b|;
* gradients and predictions against the oracle in its bfloat16-storage mode, element by
  element: the two differ by FP32 vs FP64 accumulation (K 2^-24 of the absolute sum of
  each product) and by the rare value that sits on a bfloat16 rounding boundary and
  rounds the other way (one bfloat16 ulp, 2^-7 relative, of one operand). Both are bounded
  by a multiple of the element's magnitude S: the same expression evaluated on absolute
  values (|A| |B| for every product, |dsilu| for the activation derivative, and
  2 (|y| + |t|)/n, the magnitude of y - t with y's own absolute evaluation, for the output
  error). Every element stays within 2^-10 S (a few rounding flips), and all but 0.1 %
  within 2^-14 S (accumulation alone); an FP32-accumulating emulation of the GPU
  arithmetic stays below 2.5e-5 S on these inputs. Norm checks as well: 2e-3 against the
  bfloat16 mode, 5e-2 against the plain FP64 oracle (bfloat16 rounding of every operand).
"""
import os

import numpy as np
import pytest

from oracle import eos
from oracle import mlp as omlp
from paper_2301_12869_gb300 import _build, inputs, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_lib():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    if not os.path.exists(lbm.LIB_PATH):
        _build.build()
    lbm.load()


def bf16_bits(a):
    """bfloat16 bit patterns (int16 tensor on the GPU) of the bfloat16 rounding of a."""
    import torch

    r = omlp.to_bf16(a).astype(np.float32)
    bits = (r.view(np.uint32) >> 16).astype(np.uint16).view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(bits)).cuda(), r.astype(np.float64)


@pytest.mark.parametrize("M, N, K, k_split, acc", [
    (128, 128, 64, 0, False),
    (200, 128, 16, 0, False),     # ragged M, one K step
    (300, 200, 192, 0, False),    # ragged M and N (two N tiles), three K chunks through both stages
    (128, 16, 1024, 256, True),   # split K with atomic accumulation, N = 16
    (256, 128, 640, 0, False),    # ten K chunks
    (40, 24, 80, 0, False),       # one partial tile in M and N; the second chunk has one K step
    (512, 384, 4096, 1024, True), # four K splits of sixteen chunks: every stage refilled five times
    (128, 128, 1040, 0, False),   # seventeen chunks, the last one K step
])
def test_tensor_core_gemm_matches_exact_product(M, N, K, k_split, acc):
    import torch

    rng = np.random.default_rng(M + N + K)
    A, Ar = bf16_bits(rng.normal(size=(M, K)))
    B, Br = bf16_bits(rng.normal(size=(N, K)))
    C0 = rng.normal(size=(M, N)).astype(np.float32) if acc else np.zeros((M, N), np.float32)
    C = torch.from_numpy(C0.copy()).cuda()
    lbm.lbm_mlp_gemm(A, B, C, k_split=k_split, accumulate=acc)
    want = Ar @ Br.T + (C0 if acc else 0.0)
    bound = 2 * K * 2.0**-24 * (np.abs(Ar) @ np.abs(Br).T) + 1e-6 * np.abs(C0)
    assert np.all(np.abs(C.cpu().numpy() - want) <= bound + 1e-30)


def test_enqueued_gemm_replays_in_a_cuda_graph():
    """lbm_mlp_gemm_enqueue allocates and waits for nothing: captured once in a CUDA graph
    with the accumulating epilogue, each replay adds A B^T to C again; the status word stays 0."""
    import torch

    M, N, K = 384, 256, 320
    rng = np.random.default_rng(17)
    A, Ar = bf16_bits(rng.normal(size=(M, K)))
    B, Br = bf16_bits(rng.normal(size=(N, K)))
    C = torch.zeros(M, N, device="cuda", dtype=torch.float32)
    status = torch.zeros(1, device="cuda", dtype=torch.int32)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        lbm.lbm_mlp_gemm_enqueue(A, B, C, status, accumulate=True, stream=s.cuda_stream)  # eager, before capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        lbm.lbm_mlp_gemm_enqueue(A, B, C, status, accumulate=True, stream=s.cuda_stream)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    want = 4.0 * (Ar @ Br.T)
    bound = 4 * 2 * K * 2.0**-24 * (np.abs(Ar) @ np.abs(Br).T) + 4 * 2.0**-22 * np.abs(want)
    assert np.all(np.abs(C.cpu().numpy() - want) <= bound + 1e-30)
    assert int(status.item()) == 0
    with pytest.raises(lbm.LbmError, match="multiple of 16"):
        lbm.lbm_mlp_gemm_enqueue(A[:, :24].contiguous(), B[:, :24].contiguous(), C, status)


def params_for_test(seed=1):
    P = omlp.init_params(inputs.mlp_draws(seed))
    rng = np.random.default_rng(seed)
    for k in ("b1", "b2", "b3"):
        P[k] = 0.2 * (rng.random(128) - 0.5)
    P["b4"] = np.array([0.7])
    return P


def features(n, seed):
    rng = np.random.default_rng(seed)
    raw = np.column_stack([rng.uniform(0.7, 0.95, n), rng.uniform(-6, -4, n), rng.integers(1, 3, n),
                           rng.uniform(0.3, 2.5, n), rng.random(n), rng.integers(6, 11, n)])
    t = 1.3 - 1.0 * np.tanh(8.0 * (raw[:, 4] - 0.5)) + 0.2 * (raw[:, 0] - 0.8)
    return raw.astype(np.float32), t.astype(np.float32)


def to_gpu(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_err(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-30)


def magnitudes(x, t, P):
    """Magnitude S of every gradient element and of every prediction for the bfloat16-mode
    network: each quantity re-evaluated with every operand replaced by its absolute value
    (and bfloat16-rounded where the network rounds it). |silu(z)| <= |z| bounds the
    activations; the output error y - t has magnitude |y|_abs + |t|."""
    r, A = omlp.to_bf16, np.abs
    _, c = omlp.forward(x, P, bf16=True)
    n = len(t)
    aY = A(c["H3"]) @ A(P["w4"]) + A(P["b4"][0])
    ady = 2.0 * (aY + A(t)) / n
    gZ3 = np.outer(ady, A(P["w4"])) * A(omlp.dsilu(c["Z3"]))
    gZ2 = (gZ3 @ A(r(P["W3"]))) * A(omlp.dsilu(c["Z2"]))
    gZ1 = (gZ2 @ A(r(P["W2"]))) * A(omlp.dsilu(c["Z1"]))
    S = {"w4": A(c["H3"]).T @ ady, "b4": np.array([ady.sum()]),
         "W3": gZ3.T @ A(r(c["H2"])), "b3": gZ3.sum(axis=0),
         "W2": gZ2.T @ A(r(c["H1"])), "b2": gZ2.sum(axis=0),
         "W1": gZ1.T @ A(c["X"]), "b1": gZ1.sum(axis=0)}
    return S, aY


def assert_elementwise(got, want, S, what):
    """|got - want| <= 2^-10 S everywhere, <= 2^-14 S on all but 0.1 % of the elements."""
    d = np.abs(np.asarray(got, dtype=np.float64) - want)
    ratio = d / np.maximum(S, 1e-300)
    assert np.all(d <= 2.0**-10 * S + 1e-30), (what, float(ratio.max()), np.unravel_index(np.argmax(ratio), d.shape))
    assert np.mean(ratio > 2.0**-14) <= 1e-3, (what, float(np.mean(ratio > 2.0**-14)))


@pytest.mark.parametrize("n", [128, 300])
def test_gradients_match_oracle(n):
    P = params_for_test()
    raw, t = features(n, 5)
    h = lbm.lbm_mlp_create(lbm.mlp_pack(P), 384)
    try:
        # the oracle sees what the network sees: FP32 parameters and FP32 feature rows
        Pf = lbm.mlp_unpack(lbm.lbm_mlp_get_params(h))
        x = omlp.normalise(raw.astype(np.float64)).astype(np.float32).astype(np.float64)
        loss, g = lbm.lbm_mlp_gradients(h, to_gpu(raw), to_gpu(t))
        G = lbm.mlp_unpack(g)
        assert np.all(g[:128 * 16].reshape(128, 16)[:, lbm.MLP_INPUTS:] == 0)  # padded inputs get no gradient
        l16, g16 = omlp.loss_and_grads(x, t.astype(np.float64), Pf, bf16=True)
        l64, g64 = omlp.loss_and_grads(x, t.astype(np.float64), Pf)
        S, _ = magnitudes(x, t.astype(np.float64), Pf)
        assert loss == pytest.approx(l16, rel=2e-3)
        for k in g16:
            assert_elementwise(G[k], g16[k], S[k], k)
            assert rel_err(G[k], g16[k]) <= 2e-3, k
            assert rel_err(G[k], g64[k]) <= 5e-2, k
    finally:
        lbm.lbm_mlp_destroy(h)


def test_prediction_matches_oracle():
    import torch

    P = params_for_test(2)
    raw, _ = features(1000, 6)  # three passes of 384 rows, the last one partial
    h = lbm.lbm_mlp_create(lbm.mlp_pack(P), 384)
    try:
        Pf = lbm.mlp_unpack(lbm.lbm_mlp_get_params(h))
        y = torch.empty(1000, dtype=torch.float32, device="cuda")
        lbm.lbm_mlp_predict(h, to_gpu(raw), y)
        x = omlp.normalise(raw.astype(np.float64)).astype(np.float32).astype(np.float64)
        want, _ = omlp.forward(x, Pf, bf16=True)
        _, aY = magnitudes(x, np.zeros(len(x)), Pf)
        assert_elementwise(y.cpu().numpy(), want, aY, "prediction")
        assert rel_err(y.cpu().numpy(), want) <= 2e-3
    finally:
        lbm.lbm_mlp_destroy(h)


def test_fused_forward_over_many_tiles():
    """lbm_mlp_predict runs the fused forward kernel: persistent CTAs with two 128-row tile
    pipelines each. 303 tiles (the last one 77 rows) give every CTA several tiles and its
    two groups different counts; sampled rows (the first and last tiles whole, 1500 random)
    against the oracle in its bfloat16 mode, element-wise as above."""
    import torch

    P = params_for_test(5)
    n = 128 * 302 + 77
    raw, _ = features(n, 9)
    h = lbm.lbm_mlp_create(lbm.mlp_pack(P), 256)
    try:
        Pf = lbm.mlp_unpack(lbm.lbm_mlp_get_params(h))
        y = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        lbm.lbm_mlp_predict(h, to_gpu(raw), y)
        got = y.cpu().numpy()
        assert np.all(np.isfinite(got))  # every row written
        rng = np.random.default_rng(3)
        rows = np.unique(np.concatenate([np.arange(128), np.arange(n - 77, n), rng.integers(0, n, 1500)]))
        x = omlp.normalise(raw[rows].astype(np.float64)).astype(np.float32).astype(np.float64)
        want, _ = omlp.forward(x, Pf, bf16=True)
        _, aY = magnitudes(x, np.zeros(len(x)), Pf)
        assert_elementwise(got[rows], want, aY, "fused forward")
    finally:
        lbm.lbm_mlp_destroy(h)


def test_adam_steps_match_oracle():
    """Three training steps with the SplitMix64 minibatches of the input module: the
    parameters follow the oracle's Adam (bfloat16 mode) to a small fraction of lr."""
    P = params_for_test(3)
    raw, t = features(500, 7)
    lr, batch, seed = 1e-3, 256, 99
    h = lbm.lbm_mlp_create(lbm.mlp_pack(P), 256)
    try:
        Pf = lbm.mlp_unpack(lbm.lbm_mlp_get_params(h))
        losses = lbm.lbm_mlp_train(h, to_gpu(raw), to_gpu(t), batch, 3, lr, seed)
        Pg = lbm.mlp_unpack(lbm.lbm_mlp_get_params(h))
        x = omlp.normalise(raw.astype(np.float64)).astype(np.float32).astype(np.float64)
        Po = Pf
        m = {k: np.zeros_like(v) for k, v in Po.items()}
        v = {k: np.zeros_like(v) for k, v in Po.items()}
        for step in range(3):
            idx = inputs.minibatch_indices(500, batch, step, seed)
            lo, g = omlp.loss_and_grads(x[idx], t[idx].astype(np.float64), Po, bf16=True)
            assert losses[step] == pytest.approx(lo, rel=5e-3)
            Po, m, v = omlp.adam_step(Po, g, m, v, step + 1, lr=lr)
        for k in Po:
            d = np.abs(Pg[k] - Po[k]).ravel()
            # a component whose gradient is within rounding of zero may take the opposite sign
            assert np.mean(d > 0.1 * lr) <= 0.01, k
            assert np.max(d) <= 6 * lr, k
    finally:
        lbm.lbm_mlp_destroy(h)


def test_training_lowers_the_loss():
    raw, t = features(4096, 8)
    h = lbm.lbm_mlp_create(lbm.mlp_pack(params_for_test(4)), 512)
    try:
        losses = lbm.lbm_mlp_train(h, to_gpu(raw), to_gpu(t), 512, 300, 3e-3, 1)
        assert np.all(np.isfinite(losses))
        assert np.mean(losses[-20:]) < 0.05 * np.mean(losses[:5])
    finally:
        lbm.lbm_mlp_destroy(h)


def test_features_and_warm_start_profile():
    import torch

    a, b, R = 0.25, 4.0, 1.0
    rho_c, T_c, _ = eos.critical_point(a, b, R)
    cols = [dict(ny=64, T=0.8 * T_c, gy=-1e-5, form=1), dict(ny=128, T=0.9 * T_c, gy=-3e-6, form=2),
            dict(ny=16, T=0.75 * T_c, gy=-1e-4, form=1)]
    mean = np.array([0.12, 0.15, 0.2])
    nx = 4
    rows = sum(c["ny"] for c in cols)
    x = torch.empty((rows, lbm.MLP_INPUTS), dtype=torch.float32, device="cuda")
    lbm.lbm_mlp_features(cols, nx, a, b, R, x, mean_rho=mean)
    want = np.concatenate([np.column_stack([np.full(c["ny"], c["T"] / T_c), np.full(c["ny"], np.log10(abs(c["gy"]))),
                                            np.full(c["ny"], c["form"]), np.full(c["ny"], m / rho_c),
                                            (np.arange(c["ny"]) + 0.5) / c["ny"], np.full(c["ny"], np.log2(c["ny"]))])
                           for c, m in zip(cols, mean)])
    np.testing.assert_allclose(x.cpu().numpy(), want, rtol=1e-6)
    h = lbm.lbm_mlp_create(lbm.mlp_pack(params_for_test(5)), 128)
    try:
        rho0 = torch.empty(nx * rows, dtype=torch.float64, device="cuda")
        lbm.lbm_mlp_warm_start(h, cols, nx, a, b, R, mean, rho0)
        r = rho0.cpu().numpy()
        y = torch.empty(rows, dtype=torch.float32, device="cuda")
        lbm.lbm_mlp_predict(h, x, y)
        yh = y.cpu().numpy().astype(np.float64)
        off = roff = 0
        for c, m in zip(cols, mean):
            ny = c["ny"]
            blk = r[off:off + nx * ny].reshape(ny, nx)
            off += nx * ny
            assert np.all(blk == blk[:, :1])              # the same on every x
            assert blk.mean() == pytest.approx(m, rel=1e-12)  # mass of the column kept exactly
            assert np.all(blk > 0)
            # the predicted profile moved along y to the column's mass (the stated definition)
            prof = np.maximum(yh[roff:roff + ny] * rho_c, 1e-3)
            roff += ny
            moved = lambda s: np.interp(np.arange(ny) - s, np.arange(ny), prof)  # noqa: E731
            lo, hi, target = -ny, ny, m * ny
            shift = 0.0
            if moved(lo).sum() <= target <= moved(hi).sum():
                for _ in range(60):
                    mid = 0.5 * (lo + hi)
                    lo, hi = (mid, hi) if moved(mid).sum() < target else (lo, mid)
                shift = 0.5 * (lo + hi)
            want_col = moved(shift) * target / moved(shift).sum()
            np.testing.assert_allclose(blk[:, 0], want_col, rtol=1e-9, atol=0)
        # features from the columns' own density fields: <rho> from the field, targets rho/rho_c
        t = torch.empty(rows, dtype=torch.float32, device="cuda")
        lbm.lbm_mlp_features(cols, nx, a, b, R, x, t=t, rho=rho0)
        np.testing.assert_allclose(x.cpu().numpy()[:, 3], want[:, 3], rtol=1e-6)
        np.testing.assert_allclose(t.cpu().numpy(), r.reshape(-1, nx)[:, 0] / rho_c, rtol=1e-6)
    finally:
        lbm.lbm_mlp_destroy(h)


def test_warm_start_gain_on_held_out_columns():
    """What the trained network gains over the method without it, on held-out columns:
    trained on the steady profiles of 4096 seeded 4 x 64 columns (FP32 runs of the method;
    8000 Adam steps of 8192 rows - a network trained on a few hundred columns for 1500 steps
    started the rest-state runs farther from the steady state than the tanh profile),
    its start is closer to the converged profile than the tanh start; the lattice Boltzmann
    run from it reaches the tanh start's steady state on most columns (the network only
    initialises; the FP64 run to 1e-10 decides); and started from the rest state of each
    profile (lbm_batch_rest_state) the network's columns need fewer steps in total than the
    tanh columns, and both far fewer than the method's own equilibrium start from tanh. (From
    equilibrium populations f_eq(rho, 0) no density profile, not even the converged one,
    saves more than ~1.5 % of the steps: the transient of the missing forcing terms sets them.)"""
    import torch

    a, b, R = 0.25, 4.0, 1.0
    rho_c, T_c, _ = eos.critical_point(a, b, R)

    def columns(n, seed):
        gen = [c for c in inputs.batched_columns(8 * n, seed=seed) if c["ny"] == 64][:n]
        cols, rhos = [], []
        for c in gen:
            rv, rl, _ = eos.maxwell(c["Tr"] * T_c, a, b, R)
            rhos.append(inputs.column_rho0(4, 64, rl, rv, max(1, int(round(c["liquid_fraction"] * 64)))))
            cols.append(dict(ny=64, T=c["Tr"] * T_c, gy=c["gy"], form=c["form"]))
        return cols, np.concatenate([r.ravel() for r in rhos])

    p32 = lbm.make_params(4, 8, 0.8 * T_C_of(a, b, R), "fp32", a=a)
    p64 = lbm.make_params(4, 8, 0.8 * T_C_of(a, b, R), "fp64", a=a)
    cols, rho = columns(4096, 11)
    bt = lbm.lbm_batch_init(p32, cols, rho)
    lbm.lbm_batch_run(bt, 1e-7, 100000, 100)
    _, res, status = lbm.lbm_batch_results(bt, len(cols), check=False)
    rho_dev = torch.empty(rho.size, dtype=torch.float64, device="cuda")
    lbm.lbm_batch_moments(bt, rho=rho_dev)
    lbm.lbm_batch_destroy(bt)
    x = torch.empty((64 * len(cols), lbm.MLP_INPUTS), dtype=torch.float32, device="cuda")
    t = torch.empty(64 * len(cols), dtype=torch.float32, device="cuda")
    lbm.lbm_mlp_features(cols, 4, a, b, R, x, t=t, rho=rho_dev)
    keep = torch.from_numpy(np.repeat((res <= 1e-7) & (status == 0), 64)).cuda()
    h = lbm.lbm_mlp_create(lbm.mlp_initial_params(3), 8192)
    try:
        xk, tk = x[keep].contiguous(), t[keep].contiguous()
        for k, (iters, lr) in enumerate(((4000, 1e-3), (2400, 3e-4), (1600, 1e-4))):
            lbm.lbm_mlp_train(h, xk, tk, 8192, iters, lr, 5 + k, record=False)
        ev, rho0 = columns(256, 12)
        mean = rho0.reshape(len(ev), -1).mean(axis=1)
        warm = torch.empty(rho0.size, dtype=torch.float64, device="cuda")
        lbm.lbm_mlp_warm_start(h, ev, 4, a, b, R, mean, warm)
    finally:
        lbm.lbm_mlp_destroy(h)
    runs = {}
    for name, start, rest in (("tanh", rho0, False), ("warm", warm, False), ("tanh_rest", rho0, True),
                              ("warm_rest", warm, True)):
        bb = lbm.lbm_batch_init(p64, ev, start)
        if rest:
            lbm.lbm_batch_rest_state(bb)
        lbm.lbm_batch_run(bb, 1e-10, 200000, 100)
        steps, res, status = lbm.lbm_batch_results(bb, len(ev), check=False)
        f = np.empty(rho0.size)
        lbm.lbm_batch_moments(bb, rho=f)
        lbm.lbm_batch_destroy(bb)
        runs[name] = (f, (res <= 1e-10) & (status == 0), steps)
    ok = np.logical_and.reduce([r[1] for r in runs.values()])
    assert ok.sum() >= 0.8 * len(ev)
    per = lambda v: np.abs(v).reshape(len(ev), -1).max(axis=1)  # noqa: E731
    ref = runs["tanh"][0]
    err_tanh = per(rho0 - ref)[ok]
    err_warm = per(warm.cpu().numpy() - ref)[ok]
    assert np.median(err_warm) < np.median(err_tanh)
    # a column's steady state need not be unique: a start can settle in another basin (a
    # "miss", which only the plain run reveals). Runs stopped at a per-step change of 1e-10
    # are within 1e-10 / (1 - r) of their fixed point, r the per-step decay factor of the
    # slowest mode (1 - r ~ 5e-4 here): same state = within 1e-5. Most columns agree.
    same = per(runs["warm_rest"][0] - ref)[ok] <= 1e-5
    assert np.mean(same) >= 0.9
    total = {k: int(v[2][ok].sum()) for k, v in runs.items()}
    per_col = runs["warm_rest"][2][ok] / runs["tanh_rest"][2][ok]
    # measured: totals 0.958 (warm / tanh, rest-state starts) and 0.80 (against the plain
    # method); per column median 0.945, 62 % of the columns faster
    assert total["warm_rest"] < 0.97 * total["tanh_rest"], total
    assert total["warm_rest"] < 0.85 * total["tanh"], total
    assert np.median(per_col) < 0.99 and np.mean(per_col < 1.0) > 0.5


def T_C_of(a, b, R):
    return eos.critical_point(a, b, R)[1]
