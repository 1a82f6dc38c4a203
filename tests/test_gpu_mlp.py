"""The warm-start network's GPU kernels against the oracle (oracle/mlp.py), and the
learned warm start against the method without it.

Parity tolerances: the GPU computes in FP32 with the same bfloat16-rounded weights as
the oracle (which computes in FP64), so forward outputs agree to FP32 rounding over
sums of <= 256 terms (1e-5 relative to the output scale) and gradients to 1e-4 of each
tensor's largest entry (sums over all samples).  The products of the 256-input layers run
on the tensor cores by default (each FP32 activation as three bfloat16 terms, FP32
accumulation): the same tolerances hold, and the CUDA-core products are checked too."""
import numpy as np
import pytest

import absorber_inputs as ai
from oracle import checks, mlp

pytestmark = pytest.mark.gpu
P = ai.PARAMS


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_15420_gb300 import build
    build.build()
    from paper_2607_15420_gb300 import binding
    binding.lib()
    return binding


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _case(seed, n):
    rng = np.random.default_rng(seed)
    parts = []
    for s in mlp.SHAPES:
        fan_in = s[1] if len(s) == 2 else 1
        parts.append(rng.normal(0, 1.0 / np.sqrt(fan_in), s))
    theta = _f32(mlp.flatten(parts))
    norm = dict(in_shift=_f32(rng.normal(0, 0.2, mlp.N_IN)), in_scale=_f32(rng.uniform(0.5, 2.0, mlp.N_IN)),
                out_shift=_f32(rng.normal(0, 1, mlp.N_OUT)), out_scale=_f32(rng.uniform(0.5, 2.0, mlp.N_OUT)))
    X = _f32(rng.normal(0, 1, (n, mlp.N_IN)))
    Y = _f32(rng.normal(0, 1, (n, mlp.N_OUT)))
    return theta, norm, X, Y


def _net(B, theta, norm):
    net = B.MLP(seed=3)
    net.set_params(theta)
    net.set_normalization(norm["in_shift"], norm["in_scale"], norm["out_shift"], norm["out_scale"])
    return net


def _dev32(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n", [1, 77, 300])
def test_forward_matches_oracle(B, n):
    import torch
    theta, norm, X, Y = _case(10 + n, n)
    net = _net(B, theta, norm)
    Yg = torch.zeros((n, mlp.N_OUT), dtype=torch.float32, device="cuda")
    net.forward(_dev32(X), Yg)
    yo = mlp.predict(theta, X, norm)
    scale = norm["out_scale"] * (1.0 + np.abs(mlp.forward(theta, X, norm)))
    assert np.max(np.abs(_host(Yg) - yo) / scale) <= 1e-5


@pytest.mark.parametrize("n", [128, 300, 5000])
def test_tensor_core_products_match_cuda_core_products_and_oracle(B, n):
    # the tcgen05 forward products (tiles of 128 rows x 64 columns; 440 outputs = 6 full
    # tiles and a 56-column one; ragged last row tile) against the FP32 FMA products and
    # the oracle; no wait gave up
    import torch
    theta, norm, X, Y = _case(40 + n, n)
    net = _net(B, theta, norm)
    Yt = torch.zeros((n, mlp.N_OUT), dtype=torch.float32, device="cuda")
    Yc = torch.zeros_like(Yt)
    net.forward(_dev32(X), Yt)
    net.set_tensor_cores(0)
    net.forward(_dev32(X), Yc)
    net.set_tensor_cores(1)
    yt, yc = _host(Yt), _host(Yc)
    assert net.device_fault() == 0
    rows = np.arange(n) if n <= 300 else np.r_[0:64, 2500:2564, n - 72:n]
    yo = mlp.predict(theta, X[rows], norm)
    scale = norm["out_scale"] * (1.0 + np.abs(mlp.forward(theta, X[rows], norm)))
    assert np.max(np.abs(yt[rows] - yo) / scale) <= 1e-5
    assert np.max(np.abs(yc[rows] - yo) / scale) <= 1e-5
    # every row: the two within twice that bound of each other (each within it of the
    # exact product), on the normalised-output scale
    yn = (yc - norm["out_shift"]) / norm["out_scale"]
    assert np.max(np.abs(yt - yc) / (norm["out_scale"] * (1.0 + np.abs(yn)))) <= 2e-5
    with pytest.raises(B.AbsorberError):
        net.set_tensor_cores(2)


def test_tensor_core_wait_expiry_is_reported(B):
    # the one device-side wait: its self-test withholds the MMAs so that the bounded wait
    # runs out; the kernel frees its tensor memory and reports through the fault flag, the
    # call returns ABS_ERR_TIMEOUT and clears the flag, and the products work afterwards
    import torch
    theta, norm, X, Y = _case(77, 300)
    net = _net(B, theta, norm)
    assert net.device_fault() == 0
    assert net.selftest_wait() == -8   # ABS_ERR_TIMEOUT
    assert net.device_fault() == 0
    Yt = torch.zeros((300, mlp.N_OUT), dtype=torch.float32, device="cuda")
    net.forward(_dev32(X), Yt)
    yo = mlp.predict(theta, X, norm)
    scale = norm["out_scale"] * (1.0 + np.abs(mlp.forward(theta, X, norm)))
    assert np.max(np.abs(_host(Yt) - yo) / scale) <= 1e-5
    assert net.device_fault() == 0


def test_forward_large_chunked(B):
    # more rows than one inference pass holds (8192): sampled rows against the oracle
    import torch
    n = 9000
    theta, norm, X, Y = _case(5, n)
    net = _net(B, theta, norm)
    Yg = torch.zeros((n, mlp.N_OUT), dtype=torch.float32, device="cuda")
    net.forward(_dev32(X), Yg)
    rows = np.array([0, 1, 4095, 8191, 8192, 8193, 8999])
    yo = mlp.predict(theta, X[rows], norm)
    scale = norm["out_scale"] * (1.0 + np.abs(mlp.forward(theta, X[rows], norm)))
    assert np.max(np.abs(_host(Yg)[rows] - yo) / scale) <= 1e-5


@pytest.mark.parametrize("n", [3, 130])
def test_gradient_matches_oracle(B, n):
    import torch
    theta, norm, X, Y = _case(20 + n, n)
    net = _net(B, theta, norm)
    g = torch.zeros(mlp.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = net.loss_grad(_dev32(X), _dev32(Y), grad=g)
    lo, go = mlp.loss_and_grad(theta, X, Y, norm, bf16=True)
    assert abs(loss - lo) <= 1e-5 * lo
    gg = _host(g)
    offs = np.cumsum([0] + [int(np.prod(s)) for s in mlp.SHAPES])
    for k in range(8):
        a, b = offs[k], offs[k + 1]
        err = np.max(np.abs(gg[a:b] - go[a:b]))
        assert err <= 1e-4 * np.max(np.abs(go[a:b])), (k, err, np.max(np.abs(go[a:b])))


def test_adam_step_matches_oracle(B):
    # one epoch with one full batch is exactly one Adam step from zero moments
    n = 64
    theta, norm, X, Y = _case(31, n)
    net = _net(B, theta, norm)
    lr = 1e-3
    hist = net.train(_dev32(X), _dev32(Y), B.train_options(epochs=1, batch=n, lr=lr, lr_final=lr))
    lo, go = mlp.loss_and_grad(theta, X, Y, norm, bf16=True)
    assert abs(hist[0] - lo) <= 1e-5 * lo
    th1, _, _ = mlp.adam_step(theta, go, np.zeros_like(theta), np.zeros_like(theta), 1, lr)
    tg = net.get_params().astype(np.float64)
    # the first Adam step is lr * g / (|g| + eps): entries whose gradient is within a few
    # FP32 roundings of zero may take a step of any size up to lr
    big = np.abs(go) > 1e-3 * np.max(np.abs(go))
    assert np.max(np.abs(tg - th1)[big]) <= 1e-3 * lr + 1e-7 * np.max(np.abs(theta))
    assert np.max(np.abs(tg - theta)) <= lr * (1 + 1e-5) + 1e-7 * np.max(np.abs(theta))


def test_fit_normalization(B):
    rng = np.random.default_rng(8)
    n = 1000
    X = rng.normal(3.0, 0.5, (n, mlp.N_IN)).astype(np.float32)
    Y = rng.normal(-2.0, 4.0, (n, mlp.N_OUT)).astype(np.float32)
    Y[:, 5] = 7.0                        # a constant column keeps scale 1
    net = B.MLP(seed=1)
    net.fit_normalization(_dev32(X), _dev32(Y))
    nm = net.get_normalization()
    np.testing.assert_allclose(nm["in_shift"], X.astype(np.float64).mean(0), rtol=1e-6)
    np.testing.assert_allclose(nm["in_scale"], X.astype(np.float64).std(0), rtol=1e-5)
    np.testing.assert_allclose(nm["out_shift"], Y.astype(np.float64).mean(0), rtol=1e-6, atol=1e-6)
    sd = Y.astype(np.float64).std(0)
    sd[5] = 1.0
    np.testing.assert_allclose(nm["out_scale"], sd, rtol=1e-5)


def _training_set(B, n_train, seed):
    """Solutions of n_train one-scenario problems (one batched solve from a shared
    expected-value start) as training pairs, with diameter copies."""
    import torch
    F = ai.make_feeds(n_train, seed, stream=3)
    batch = B.Batch(P, [F[:, i:i + 1] for i in range(n_train)])
    x = torch.zeros(batch.n_primal, dtype=torch.float64, device="cuda")
    y = torch.zeros(220 * batch.ld, dtype=torch.float64, device="cuda")
    # one shared expected-value start; objective scaled by 100 (the optimum does not
    # change) -- with w = 1 the barrier terms dominate and the line search stalls on
    # about one single-scenario problem in eight, in the oracle as on the GPU
    res = batch.ipm_solve(B.default_options(init=2, obj_scaling=100.0), x_out=x, y_out=y)
    keep = [r.status == 0 for r in res]
    assert sum(keep) >= 0.95 * n_train
    X, Y = B.make_dataset(batch, x, y, keep=keep, n_aug=4, d_spread=0.15)
    assert X.shape[0] == 4 * sum(keep)
    return X, Y, batch


def test_learned_warm_start_beats_cold_start(B):
    import torch
    X, Y, _ = _training_set(B, 1500, 7)
    net = B.MLP(seed=11)
    net.fit_normalization(X, Y)
    hist = net.train(X, Y, B.train_options(epochs=150, batch=250, lr=2e-3, lr_final=2e-5, seed=5))
    assert hist[-1] < 0.05 * hist[0]
    F = ai.make_feeds(400, 4)
    prob = B.Problem(P, F)
    o = B.default_options()
    cold = prob.ipm_solve(o)
    xw = torch.zeros(prob.n_primal, dtype=torch.float64, device="cuda")
    yw = torch.zeros(prob.n_row, dtype=torch.float64, device="cuda")
    warm = B.ipm_solve_learned(prob, net, o, x_out=xw, y_out=yw)
    assert cold.status == 0 and warm.status == 0
    assert warm.warm_status == 1, (warm.warm_E0, warm.cold_E0, warm.warm_theta, warm.cold_theta)
    assert warm.E0 <= 1e-8
    assert abs(warm.d - cold.d) <= 1e-6 * cold.d
    # the gain: far fewer iterations than the default start's (its own plus those of the
    # expected-value solve), and less wall time including the prediction
    assert warm.iters + warm.base_iters <= 0.5 * (cold.iters + cold.base_iters), (warm.iters, cold.iters,
                                                                                  cold.base_iters)
    assert warm.solve_ms < cold.solve_ms
    # the learned point is near the central path: its optimality error is a small fraction
    # of the inlet-copy start's
    assert warm.warm_E0 < 1e-2 * warm.cold_E0 and warm.warm_theta < warm.cold_theta
    # the multipliers the solve returns are those of the same optimum
    dmin, _ = checks.minimum_diameter(P, F, prob.from_soa(_host(xw))[0])
    assert abs(warm.d - dmin) <= 1e-8 * dmin
    # E_0 at the returned point, recomputed from the definitions by the oracle's check
    zl, zu = torch.zeros_like(xw), torch.zeros_like(xw)
    zd = prob.bound_multipliers(zl, zu)
    Z, d = prob.from_soa(_host(xw))
    lam, _ = prob.from_soa(_host(yw))
    ZL, _ = prob.from_soa(_host(zl))
    ZU, _ = prob.from_soa(_host(zu))
    assert checks.kkt_error(P, F, d, Z, lam, ZL, ZU, zd[0], zd[1], chunk=100) <= 1e-8
    # repeated solves replay the captured graphs (the inlet-copy evaluation on the second
    # handle, the solve from the learned start waiting for it): the first solve bit for bit
    again = [B.ipm_solve_learned(prob, net, o) for _ in range(3)]
    assert again[-1].graph_replays >= 1
    for r in again:
        assert r.status == 0 and r.warm_status == 1 and r.iters == warm.iters and r.d == warm.d
        assert r.warm_E0 == warm.warm_E0 and r.cold_E0 == warm.cold_E0
    # the same with FP32 factors and FP64 refinement
    o32 = B.default_options(precision=1, max_refine=8)
    w32 = [B.ipm_solve_learned(prob, net, o32) for _ in range(4)]
    assert w32[-1].graph_replays >= 1
    for r in w32:
        assert r.status == 0 and r.warm_status == 1 and r.E0 <= 1e-8 and abs(r.d - warm.d) <= 1e-6 * warm.d
        assert r.iters == w32[0].iters and r.d == w32[0].d


def test_learned_warm_start_rejects_a_bad_network(B):
    # an untrained network's start is rejected and the solve runs from the default start
    F = ai.make_feeds(20, 4)
    prob = B.Problem(P, F)
    net = B.MLP(seed=2)
    o = B.default_options()
    cold = prob.ipm_solve(o)
    warm = B.ipm_solve_learned(prob, net, o)
    assert warm.warm_status == 0 and warm.status == 0
    assert warm.iters == cold.iters and abs(warm.d - cold.d) <= 1e-12 * cold.d


def test_learned_warm_start_full_size_s20000(B):
    # the 20,000-scenario workload from the learned start with FP32 factors: the same
    # optimum as the FP64 path from the default start, in fewer iterations
    X, Y, _ = _training_set(B, 4000, 7)
    net = B.MLP(seed=11)
    net.fit_normalization(X, Y)
    net.train(X, Y, B.train_options(epochs=60, batch=256, lr=2e-3, lr_final=2e-5, seed=5))
    F = ai.workload_feeds("absorber-S20000-u10-seed4")
    prob = B.Problem(P, F)
    cold = prob.ipm_solve(B.default_options())
    warm = B.ipm_solve_learned(prob, net, B.default_options(precision=1, max_refine=8))
    assert cold.status == 0 and warm.status == 0 and warm.E0 <= 1e-8
    assert warm.warm_status == 1
    assert abs(warm.d - cold.d) <= 1e-6 * cold.d
    assert warm.iters < cold.iters + cold.base_iters
