"""Learned warm start / preconditioner: the MLP kernels against the FP64
oracle MLP (forward, gradient, loss, Adam step, features, targets), a fit
with the learned start against the oracle's learned CoFEM loop, and the gain
over plain CG on held-out problems."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from oracle import sbl
from paper_2202_12808_gb300 import api
from paper_2202_12808_gb300 import binding as B
from paper_2202_12808_gb300 import datagen
from gpu_helpers import rel_l2, support_compare

pytestmark = pytest.mark.gpu


def _weights(seed):
    th = omlp.init_params(seed) + 0.1 * np.random.default_rng(seed).standard_normal(omlp.N_PARAMS)
    return th


def _data(n, seed):
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((n, 4)).astype(np.float32)
    Y = rng.standard_normal((n, 2)).astype(np.float32)
    return U, Y


@pytest.mark.parametrize("wdt", ["f32", "bf16"])
def test_forward_grad_loss_vs_oracle(cuda_lib, wdt):
    th = _weights(1)
    if wdt == "f32":
        w = torch.from_numpy(th.astype(np.float32)).cuda()
        th_used = th.astype(np.float32).astype(np.float64)
        code = B.COFEM_F32
    else:
        w = torch.from_numpy(th.astype(np.float32)).to(torch.bfloat16).cuda()
        th_used = w.double().cpu().numpy()
        code = B.COFEM_BF16
    U, Y = _data(5000, 2)
    Ud, Yd = torch.from_numpy(U).cuda(), torch.from_numpy(Y).cuda()
    O = torch.empty((5000, 2), dtype=torch.float32, device="cuda")
    B.cofem_mlp_forward(w.data_ptr(), code, Ud.data_ptr(), 5000, O.data_ptr())
    g = torch.empty(omlp.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = torch.empty(B.cofem_mlp_train_workspace_bytes(5000), dtype=torch.uint8, device="cuda")
    B.cofem_mlp_grad(w.data_ptr(), code, Ud.data_ptr(), Yd.data_ptr(), 5000, g.data_ptr(),
                     loss.data_ptr(), ws.data_ptr(), ws.numel())
    torch.cuda.synchronize()
    U64, Y64 = U.astype(np.float64), Y.astype(np.float64)
    o_ref, _ = omlp.forward(th_used, U64)
    assert rel_l2(O.cpu().numpy(), o_ref) <= 1e-5
    assert rel_l2(g.cpu().numpy(), omlp.grad(th_used, U64, Y64)) <= 1e-4
    assert abs(loss.item() - omlp.loss(th_used, U64, Y64)) <= 1e-5 * omlp.loss(th_used, U64, Y64)
    if wdt == "bf16":
        # against the unrounded FP32 master weights: direction of the gradient
        gm = omlp.grad(th.astype(np.float32).astype(np.float64), U64, Y64)
        gg = g.cpu().numpy().astype(np.float64)
        assert gg @ gm / (np.linalg.norm(gg) * np.linalg.norm(gm)) >= 0.999
        assert rel_l2(gg, gm) <= 2e-2


def test_adam_step_vs_oracle(cuda_lib):
    th = _weights(3).astype(np.float32)
    master = torch.from_numpy(th).cuda()
    wbf = master.to(torch.bfloat16)
    m = torch.zeros_like(master)
    v = torch.zeros_like(master)
    U, Y = _data(3000, 4)
    Ud, Yd = torch.from_numpy(U).cuda(), torch.from_numpy(Y).cuda()
    ws = torch.empty(B.cofem_mlp_train_workspace_bytes(3000), dtype=torch.uint8, device="cuda")
    th_bf = wbf.double().cpu().numpy()
    g_ref = omlp.grad(th_bf, U.astype(np.float64), Y.astype(np.float64))
    B.cofem_mlp_adam_step(master.data_ptr(), m.data_ptr(), v.data_ptr(), wbf.data_ptr(),
                          Ud.data_ptr(), Yd.data_ptr(), 3000, 1, 1e-3, ws.data_ptr(), ws.numel())
    torch.cuda.synchronize()
    t_ref, m_ref, v_ref = omlp.adam_step(th.astype(np.float64), g_ref, np.zeros_like(g_ref),
                                         np.zeros_like(g_ref), 1, lr=1e-3)
    np.testing.assert_allclose(master.cpu().numpy(), t_ref, rtol=0, atol=2e-6)
    np.testing.assert_allclose(m.cpu().numpy(), m_ref, rtol=1e-4, atol=1e-9)
    assert torch.equal(wbf, master.to(torch.bfloat16))


def test_features_targets_vs_oracle(cuda_lib):
    rng = np.random.default_rng(6)
    D = 3000
    alpha = np.exp(rng.uniform(-3, 25, D))
    pn = rng.uniform(0.3, 3, D).astype(np.float32)
    beta = 1e4
    mu = rng.standard_normal(D) * 1e-2
    s = np.exp(rng.uniform(-12, 0, D))
    s[:5] = -1e-3                                   # negative estimates are clipped
    args = [torch.from_numpy(a).cuda() for a in (alpha, pn, mu, s)]
    U = torch.empty((D, 4), dtype=torch.float32, device="cuda")
    Y = torch.empty((D, 2), dtype=torch.float32, device="cuda")
    B.cofem_mlp_features(args[0].data_ptr(), args[1].data_ptr(), beta, args[2].data_ptr(),
                         args[3].data_ptr(), D, U.data_ptr())
    B.cofem_mlp_targets(args[0].data_ptr(), args[1].data_ptr(), beta, args[2].data_ptr(),
                        args[3].data_ptr(), D, Y.data_ptr())
    torch.cuda.synchronize()
    pn64 = pn.astype(np.float64)
    np.testing.assert_allclose(U.cpu().numpy(), omlp.features(alpha, pn64, beta, mu, s),
                               rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(Y.cpu().numpy(), omlp.targets(alpha, pn64, beta, mu, s),
                               rtol=1e-6, atol=1e-6)


def _conf1(seed, sigma=0.01):
    c = datagen.CONFIGS["dense-fp64-n256-d1024"]
    pr = datagen.dense_problem(c["N"], c["D"], c["n_nonzero"], sigma, seed)
    return pr, api.DenseOperator(torch.from_numpy(pr.Phi).cuda()), \
        torch.from_numpy(pr.y.astype(np.float32)).cuda()


def _trained(seeds, em=20, steps=1500):
    Us, Ys = [], []
    for sd in seeds:
        pr, op, y = _conf1(sd)
        p = api.params(vec_dtype=B.COFEM_F32, K=20, em_iters=em, cg_tol=1e-6, cg_max_iters=400,
                       seed=sd)
        U, Y = api.collect_training_data(op, y, pr.beta, p, em)
        Us.append(U)
        Ys.append(Y)
    net = api.LearnedWarmStart(seed=0)
    losses = net.train(torch.cat(Us), torch.cat(Ys), steps, lr=3e-3, batch=32768)
    assert losses[-1] < losses[10]
    return net


@pytest.fixture(scope="module")
def net(cuda_lib):
    return _trained(range(1, 9))


def test_learned_fit_matches_oracle_learned_loop(cuda_lib, net):
    # sigma 0.1 (beta 100): FP32 vs FP64 differences stay small over the
    # EM trajectory, so the two learned loops are comparable at 1e-4
    pr, op, y = _conf1(50, sigma=0.1)
    p = api.params(vec_dtype=B.COFEM_F32, K=16, em_iters=15, cg_tol=1e-5, cg_max_iters=400,
                   seed=50)
    p.mlp = net.bf16.data_ptr()
    r = api.fit(op, y, pr.beta, p)
    torch.cuda.synchronize()
    Phi = pr.Phi.astype(np.float64)
    pn2 = np.sum(Phi * Phi, axis=0).astype(np.float32).astype(np.float64)
    th = net.bf16.double().cpu().numpy()

    def predict(alpha, mu_prev, s_prev):
        o, _ = omlp.forward(th, omlp.features(alpha, pn2, pr.beta, mu_prev, s_prev))
        return omlp.predict(o, alpha, pn2, pr.beta)

    phi, phit, D = sbl.dense_dictionary(Phi)
    ra, rmu, rs, rst = sbl.cofem_learned(phi, phit, D, pr.y.astype(np.float32).astype(np.float64),
                                         pr.beta, 16, 15, 1e-5, 400, predict, seed=50)
    assert rel_l2(r.mu.cpu().numpy(), rmu) <= 1e-4
    eq, _ = support_compare(r.alpha.cpu().numpy(), ra)
    assert eq
    assert abs(sum(r.stats["cg_iters"]) - sum(rst.cg_iters)) <= 0.1 * sum(rst.cg_iters)
    assert B.cofem_last_fit_fallbacks() == sum(rst.fallbacks)


def test_learned_gain_over_plain_cg(cuda_lib, net):
    # held-out problems: same residual tolerance, fewer CG iterations, same result
    tot_plain = tot_learned = 0
    for sd in (100, 101):
        pr, op, y = _conf1(sd)
        p = api.params(vec_dtype=B.COFEM_F32, K=20, em_iters=50, cg_tol=1e-6, cg_max_iters=400,
                       seed=sd)
        rp = api.fit(op, y, pr.beta, p)
        p.mlp = net.bf16.data_ptr()
        rl = api.fit(op, y, pr.beta, p)
        torch.cuda.synchronize()
        assert B.cofem_last_fit_fallbacks() == 0
        assert max(rl.stats["relres"]) < 1e-6
        assert rel_l2(rl.mu.cpu().numpy(), rp.mu.cpu().numpy()) <= 1e-4
        tot_plain += sum(rp.stats["cg_iters"])
        tot_learned += sum(rl.stats["cg_iters"])
    assert tot_learned <= 0.75 * tot_plain, (tot_learned, tot_plain)


def test_untrustworthy_prediction_falls_back_to_plain_cg(cuda_lib):
    # a network whose s_hat is e^40 / c_d starts every learned solve from a
    # residual ~1e15 times ||B||: neither FP32 nor FP64 can bring it below the
    # tolerance, so every E-step after the first hits the cap and reruns as
    # plain CG from zero (in the GPU fit and in the oracle's learned loop)
    th = np.zeros(omlp.N_PARAMS)
    omlp.unpack(th)["b3"][:] = [0.0, 10.0]
    w = torch.from_numpy(th).to(torch.bfloat16).cuda()
    pr, op, y = _conf1(60, sigma=0.1)
    em, cap = 4, 150
    p = api.params(vec_dtype=B.COFEM_F32, K=16, em_iters=em, cg_tol=1e-5, cg_max_iters=cap,
                   seed=60)
    rp = api.fit(op, y, pr.beta, p)
    p.mlp = w.data_ptr()
    rl = api.fit(op, y, pr.beta, p)
    torch.cuda.synchronize()
    assert B.cofem_last_fit_fallbacks() == em - 1
    assert rl.stats["cg_iters"][0] == rp.stats["cg_iters"][0]
    for t in range(1, em):
        assert rl.stats["cg_iters"][t] == cap + rp.stats["cg_iters"][t]
    assert rel_l2(rl.mu.cpu().numpy(), rp.mu.cpu().numpy()) <= 1e-6
    Phi = pr.Phi.astype(np.float64)
    pn2 = np.sum(Phi * Phi, axis=0).astype(np.float32).astype(np.float64)

    def predict(alpha, mu_prev, s_prev):
        o, _ = omlp.forward(th, omlp.features(alpha, pn2, pr.beta, mu_prev, s_prev))
        return omlp.predict(o, alpha, pn2, pr.beta)

    phi, phit, D = sbl.dense_dictionary(Phi)
    ra, rmu, rs, rst = sbl.cofem_learned(phi, phit, D, pr.y.astype(np.float32).astype(np.float64),
                                         pr.beta, 16, em, 1e-5, cap, predict, seed=60)
    assert rst.fallbacks == [0] + [1] * (em - 1)
    assert rel_l2(rl.mu.cpu().numpy(), rmu) <= 1e-4


# ------------------------------------ learned start on the tensor cores

def _oracle_learned(Phi, y, beta, K, em, tol, cap, th, seed):
    pn2 = np.sum(Phi * Phi, axis=0).astype(np.float32).astype(np.float64)

    def predict(alpha, mu_prev, s_prev):
        o, _ = omlp.forward(th, omlp.features(alpha, pn2, beta, mu_prev, s_prev))
        return omlp.predict(o, alpha, pn2, beta)

    phi, phit, D = sbl.dense_dictionary(Phi)
    return sbl.cofem_learned(phi, phit, D, y, beta, K, em, tol, cap, predict, seed=seed)


def test_learned_fit_tensor_core_bf16(cuda_lib, net):
    """The learned start with a BF16 dictionary on the tensor cores (P's BF16
    terms written by the warm-start initialisation and the preconditioned
    direction update) against the oracle's learned loop on the BF16-rounded
    dictionary (reading R12)."""
    pr = datagen.dense_problem(256, 1024, 51, 0.1, 51)
    t16 = torch.from_numpy(pr.Phi).to(torch.bfloat16)
    Phi64 = t16.double().numpy()
    op = api.DenseOperator(t16.cuda())
    y32 = pr.y.astype(np.float32)
    p = api.params(vec_dtype=B.COFEM_F32, K=16, em_iters=15, cg_tol=1e-5, cg_max_iters=400,
                   seed=51)
    p.mlp = net.bf16.data_ptr()
    r = api.fit(op, torch.from_numpy(y32).cuda(), pr.beta, p)
    torch.cuda.synchronize()
    ra, rmu, rs, rst = _oracle_learned(Phi64, y32.astype(np.float64), pr.beta, 16, 15, 1e-5, 400,
                                       net.bf16.double().cpu().numpy(), 51)
    assert rel_l2(r.mu.cpu().numpy(), rmu) <= 1e-4
    eq, _ = support_compare(r.alpha.cpu().numpy(), ra)
    assert eq
    assert abs(sum(r.stats["cg_iters"]) - sum(rst.cg_iters)) <= 0.1 * sum(rst.cg_iters)
    assert B.cofem_last_fit_fallbacks() == sum(rst.fallbacks)


SIZES = [128, 150, 300, 511, 640, 1000]


def _batch(sigma=0.1, seed0=7):
    phis, ys, betas, seeds, refs = [], [], [], [], []
    for i, N in enumerate(SIZES):
        prob = datagen.dense_problem(N, 4 * N, max(1, N // 5), sigma, seed=seed0 + i)
        t16 = torch.from_numpy(prob.Phi).to(torch.bfloat16)
        y32 = prob.y.astype(np.float32)
        phis.append(t16.cuda())
        ys.append(torch.from_numpy(y32).cuda())
        betas.append(prob.beta)
        seeds.append(2000 + i)
        refs.append((t16.double().numpy(), y32.astype(np.float64), prob.beta))
    return phis, ys, betas, seeds, refs


def test_batched_learned_matches_oracle_learned_loop(cuda_lib, net):
    """The combined form: learned start + BF16 tensor cores + batching.  Six
    problems of uneven size in one batched fit with the network, each against
    the oracle's learned loop on its own BF16-rounded dictionary; fallback
    counts equal in total."""
    phis, ys, betas, seeds, refs = _batch()
    em, K, tol = 15, 16, 1e-5
    p = api.params(vec_dtype=B.COFEM_F32, K=K, em_iters=em, cg_tol=tol, cg_max_iters=400)
    p.mlp = net.bf16.data_ptr()
    alphas, mus, ss, st = api.fit_batched(phis, ys, betas, seeds, p)
    torch.cuda.synchronize()
    fb = B.cofem_last_fit_fallbacks()
    th = net.bf16.double().cpu().numpy()
    ofb = 0
    for i, (Phi64, y64, beta) in enumerate(refs):
        ra, rmu, rs, rst = _oracle_learned(Phi64, y64, beta, K, em, tol, 400, th, seeds[i])
        ofb += sum(rst.fallbacks)
        assert rel_l2(mus[i].cpu().numpy(), rmu) <= 1e-4, (i, rel_l2(mus[i].cpu().numpy(), rmu))
        eq, border = support_compare(alphas[i].cpu().numpy(), ra)
        assert eq, (i, border)
        tot_b, tot_o = sum(st["cg_iters"][i]), sum(rst.cg_iters)
        assert abs(tot_b - tot_o) <= 0.1 * tot_o, (i, tot_b, tot_o)
    assert fb == ofb


def test_batched_learned_fallback_equals_plain_batched(cuda_lib):
    """A network that cannot be trusted (s_hat = e^40 / c_d): from the second
    E-step on every problem's learned solve hits the cap and is rerun as
    plain CG from zero, so the batched fit returns the plain batched fit's
    results with cap + plain iterations per E-step."""
    th = np.zeros(omlp.N_PARAMS)
    omlp.unpack(th)["b3"][:] = [0.0, 10.0]
    w = torch.from_numpy(th).to(torch.bfloat16).cuda()
    phis, ys, betas, seeds, refs = _batch()
    em, cap = 4, 150
    p = api.params(vec_dtype=B.COFEM_F32, K=16, em_iters=em, cg_tol=1e-5, cg_max_iters=cap)
    ap, mp, sp, stp = api.fit_batched(phis, ys, betas, seeds, p)
    p.mlp = w.data_ptr()
    al, ml, sl, stl = api.fit_batched(phis, ys, betas, seeds, p)
    torch.cuda.synchronize()
    assert B.cofem_last_fit_fallbacks() == (em - 1) * len(phis)
    for i in range(len(phis)):
        assert stl["cg_iters"][i][0] == stp["cg_iters"][i][0]
        for t in range(1, em):
            assert stl["cg_iters"][i][t] == cap + stp["cg_iters"][i][t], (i, t)
        assert torch.equal(ml[i], mp[i]) and torch.equal(al[i], ap[i]), i
