"""Row a7: the learned support proposal (MLP forward/backward/Adam on tcgen05 BF16,
top-2s proposal, restricted OMP, fallback) against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import mlp as P
from oracle import omp as oomp
from paper_2605_30396_gb300 import synth

pytestmark = pytest.mark.gpu


def bf16(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def _params(K, seed, scale=1.0):
    p = synth.mlp_params(K, seed)
    return {k: v * (scale if k.startswith("W") else 1.0) for k, v in p.items()}


def _oracle_params_bf16(p):
    """The GPU multiplies BF16 copies of the weights (biases stay FP32)."""
    return {k: (bf16(v) if k.startswith("W") else np.asarray(v, dtype=np.float64)) for k, v in p.items()}


def _top_m(z, m):
    """The first m atoms of each row of logits z by decreasing logit, equal
    logits by smaller index: the selection rule itself, applied to the
    kernel's own logits (a validity check of the selection, not parity)."""
    K = z.shape[1]
    order = np.lexsort((np.broadcast_to(np.arange(K), z.shape), -z), axis=1)
    return order[:, :m]


def _pack64(params, K):
    """The C ABI's parameter layout (W1 padded to 64 input columns) in FP64."""
    W1 = np.zeros((256, 64))
    W1[:, :params["W1"].shape[1]] = params["W1"]
    return np.concatenate([np.ravel(W1), np.ravel(params["b1"]), np.ravel(params["W2"]), np.ravel(params["b2"]),
                           np.ravel(params["W3"]), np.ravel(params["b3"])])


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30), a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("B,K", [(1, 64), (300, 256), (1000, 1024)])
def test_forward_matches_oracle(lib, B, K):
    p = _params(K, 1)
    X = synth.signals(B, synth.hidden_dictionary(K, 2), 4, 3)
    net = lib.MLP(K, p)
    z = net.forward(torch.from_numpy(X)).cpu().numpy()
    xn = bf16(P.normalise_input(X))
    po = _oracle_params_bf16(p)
    ref = P.forward(po, xn)["z3"]
    rel, cos = _rel(z, ref)
    assert rel < 1e-2 and cos > 0.9999, (rel, cos)


@pytest.mark.parametrize("B,K,s", [(256, 128, 4), (2048, 1024, 8)])
def test_gradients_match_oracle(lib, B, K, s):
    p = _params(K, 4)
    Dh = synth.hidden_dictionary(K, 5)
    X = synth.signals(B, Dh, s, 6)
    rng = np.random.default_rng(7)
    idx = synth.distinct_supports(rng, B, K, s)
    nnz = rng.integers(1, s + 1, B)
    net = lib.MLP(K, p)
    g, loss = net.gradients(torch.from_numpy(X), torch.from_numpy(idx.astype(np.int16)).cuda(),
                            torch.from_numpy(nnz.astype(np.uint8)).cuda())
    gd = lib.mlp_unpack(g, K)
    po = _oracle_params_bf16(p)
    Y = P.support_targets(idx, nnz, K)
    xn = bf16(P.normalise_input(X))
    # the oracle's backward with the same BF16 weights and input (eps-free normalise)
    po_x = dict(po)
    gref, f = P.backward(po_x, xn, Y)
    lref = float(P.bce_with_logits(f["z3"], Y).mean())
    assert abs(loss - lref) <= 1e-3 * abs(lref)
    for k in ("W3", "b3", "W2", "b2", "W1", "b1"):
        got = gd[k][:, :45] if k == "W1" else gd[k]
        rel, cos = _rel(got, gref[k])
        assert rel < 2e-2 and cos > 0.999, (k, rel, cos)
    # the padding columns of W1 get no gradient
    assert np.abs(gd["W1"][:, 45:]).max() == 0.0


def test_adam_step_matches_oracle(lib):
    K, B, s = 128, 512, 4
    p = _params(K, 8)
    X = synth.signals(B, synth.hidden_dictionary(K, 9), s, 10)
    rng = np.random.default_rng(11)
    idx = synth.distinct_supports(rng, B, K, s)
    nnz = np.full(B, s)
    net = lib.MLP(K, p)
    it = torch.from_numpy(idx.astype(np.int16)).cuda()
    nt = torch.from_numpy(nnz.astype(np.uint8)).cuda()
    before = lib.mlp_pack(p, K).numpy().astype(np.float64)  # the FP32 master weights
    net.train_step(torch.from_numpy(X), it, nt, lr=1e-3)
    after = net.params().cpu().numpy().astype(np.float64)
    # the oracle's gradient on the same BF16 weights and input, then its Adam step
    gref, _ = P.backward(_oracle_params_bf16(p), bf16(P.normalise_input(X)), P.support_targets(idx, nnz, K))
    gv = _pack64(gref, K)
    z = np.zeros_like(gv)
    ref, _, _ = P.adam_step({"p": before}, {"p": gv}, {"p": z}, {"p": z}, 1, lr=1e-3)
    # Adam's first step moves a weight by lr g / (|g| + eps), about lr sign(g):
    # compare where the gradient is clearly nonzero, so that the gradient's
    # BF16 error cannot flip its sign; elsewhere the step is at most lr
    big = np.abs(gv) > 0.1 * np.sqrt(np.mean(gv * gv))
    assert big.sum() > 0.3 * big.size
    bad = np.abs(after - ref["p"]) > 2e-6
    assert bad[big].mean() < 1e-3, bad[big].mean()
    assert np.abs(after - before).max() <= 1e-3 * (1 + 1e-4)


def test_propose_is_top_2s_of_the_logits(lib):
    K, N = 1024, 3000
    net = lib.MLP(K, _params(K, 12))
    X = torch.from_numpy(synth.signals(N, synth.hidden_dictionary(K, 13), 8, 14))
    z = net.forward(X).cpu().numpy()
    for m in (8, 16, 32):
        cand = net.propose(X, m).cpu().numpy().view(np.uint16).astype(np.int64)
        np.testing.assert_array_equal(cand, _top_m(z, m))


@pytest.mark.parametrize("K,N,m", [(300, 1000, 2), (1000, 777, 4), (256, 129, 16), (64, 1, 32),
                                   (8, 300, 16), (4096, 500, 16)])
def test_fused_propose_ragged_shapes(lib, K, N, m):
    """Blocks of 256 atoms with a ragged last block, tiles of 128 signals with a
    ragged last tile, every m; K < m leaves the trailing slots empty (0xFFFF)."""
    net = lib.MLP(K, _params(K, 40 + K))
    X = torch.from_numpy(synth.signals(N, synth.hidden_dictionary(max(K, 16), 41), 4, 42))
    z = net.forward(X).cpu().numpy()
    cand = net.propose(X, m).cpu().numpy().view(np.uint16).astype(np.int64)
    ref = _top_m(z, min(m, K))
    np.testing.assert_array_equal(cand[:, :min(m, K)], ref)
    if K < m:
        assert (cand[:, K:] == 0xFFFF).all()


def test_fused_propose_ties_and_many_tiles(lib):
    """Exactly tied logits (duplicated W3 rows and biases, in both halves of a
    block and across blocks) go to the smaller index; 60,000 signals give every
    CTA several tiles."""
    K, N, m = 640, 60_000, 16
    p = _params(K, 50)
    for a, b in ((5, 300), (130, 2), (257, 600), (129, 128), (511, 7)):
        p["W3"][b] = p["W3"][a]
        p["b3"][b] = p["b3"][a]
    net = lib.MLP(K, p)
    X = torch.from_numpy(synth.signals(N, synth.hidden_dictionary(K, 51), 4, 52)).cuda()
    z = net.forward(X).cpu().numpy()
    cand = net.propose(X, m).cpu().numpy().view(np.uint16).astype(np.int64)
    ref = _top_m(z, m)
    np.testing.assert_array_equal(cand, ref)
    # the duplicated pairs really tie and really reach the top m somewhere
    both = np.isin(ref, [5, 300]).sum(axis=1) == 2
    assert both.any()


@pytest.mark.parametrize("m,s,K", [(16, 8, 256), (8, 4, 1024), (32, 16, 512), (32, 8, 32)])
def test_restricted_omp_matches_oracle(lib, m, s, K):
    N = 2000
    D = synth.hidden_dictionary(K, 15).astype(np.float32).astype(np.float64)
    X = synth.signals(N, D, min(s, 4), 16).astype(np.float64)
    rng = np.random.default_rng(17)
    cand = np.stack([rng.choice(K, m, replace=False) for _ in range(N)])
    idx, coef, nnz, resid = lib.encode_restricted(torch.from_numpy(D), torch.from_numpy(X),
                                                  torch.from_numpy(cand.astype(np.int16)).cuda(), s)
    ref = oomp.omp_restricted(D, X, cand, s)
    gi = lib.idx_as_long(idx).cpu().numpy()
    agree = (gi == ref["idx"]).all(axis=1).mean()
    assert agree > 0.98, agree
    ok = (gi == ref["idx"]).all(axis=1)
    np.testing.assert_allclose(coef.cpu().numpy()[ok], ref["coef"][ok], rtol=1e-3, atol=1e-5)
    rg = np.sqrt(resid.cpu().numpy().astype(np.float64).sum() / (N * 45))
    ro = np.sqrt(ref["resid_sq"].sum() / (N * 45))
    assert abs(rg - ro) <= 1e-3 * ro, (rg, ro)
    if m == K:  # every atom is a candidate: restricted OMP is plain OMP
        plain = oomp.omp(D, X, s)
        np.testing.assert_array_equal(gi[ok], plain["idx"][ok])


def _trained(lib, K, s, n_train, seed, epochs=20, lr=1e-2):
    D = synth.hidden_dictionary(K, seed)
    X = synth.signals(n_train, D, s, seed + 1)
    Dt = torch.from_numpy(D.astype(np.float32)).cuda()
    Xt = torch.from_numpy(X).cuda()
    idx, coef, nnz, resid = lib.encode(Dt, Xt, s, sync=True)
    net = lib.MLP(K, synth.mlp_params(K, seed + 2))
    losses = net.train(Xt, idx, nnz, epochs=epochs, batch=1024, lr=lr)
    return D, net, losses


def test_training_reduces_loss_and_learns_supports(lib):
    K, s = 256, 4
    D, net, losses = _trained(lib, K, s, 200000, 20)
    l = losses.cpu().numpy()
    assert l[-10:].mean() < 0.6 * l[:10].mean(), (l[:10].mean(), l[-10:].mean())
    # the gain over an untrained network: recall of the OMP support in the 2s proposals
    Xv = synth.signals(4000, D, s, 99)
    Xt = torch.from_numpy(Xv).cuda()
    Dt = torch.from_numpy(D.astype(np.float32)).cuda()
    idx, _, nnz, _ = lib.encode(Dt, Xt, s, sync=True)
    sup = lib.idx_as_long(idx).cpu().numpy()
    nz = nnz.cpu().numpy()

    def recall(n):
        c = n.propose(Xt, 2 * s).cpu().numpy().view(np.uint16)
        hit = [np.isin(sup[i, :nz[i]], c[i]).mean() for i in range(len(nz)) if nz[i]]
        return float(np.mean(hit))

    fresh = lib.MLP(K, synth.mlp_params(K, 21))
    r_tr, r_0 = recall(net), recall(fresh)
    # measured: about 0.57 after training, a few percent untrained (K = 256, 2s = 8)
    assert r_tr > 0.45 and r_tr > r_0 + 0.3, (r_tr, r_0)


def test_learned_encoder_exact_and_deploy(lib):
    K, s = 256, 4
    D, net, _ = _trained(lib, K, s, 200000, 30)
    Xv = synth.signals(5000, D, s, 31)
    Xt = torch.from_numpy(Xv).cuda()
    Dt = torch.from_numpy(D.astype(np.float32)).cuda()
    _, _, _, rp = lib.encode(Dt, Xt, s, sync=True)
    # exact mode: never worse than plain OMP, and the count matches the definition
    il, cl, nl, rl, nfb = lib.encode_learned(Dt, Xt, s, net, mode="exact", sync=True)
    rp_ = rp.cpu().numpy().astype(np.float64)
    rl32 = rl.cpu().numpy().astype(np.float32)
    assert (np.sqrt(rl32) <= np.sqrt(rp.cpu().numpy().astype(np.float32)) * np.float32(1 + 1e-6)).all()
    # restricted-only residuals for the fallback count
    cand = net.propose(Xt, 2 * s)
    _, _, _, rr = lib.encode_restricted(Dt, Xt, cand, s)
    # the fallback decision is taken in FP32 on both sides (sqrt, then x (1 + 1e-6))
    rr32 = rr.cpu().numpy().astype(np.float32)
    rp32 = rp.cpu().numpy().astype(np.float32)
    worse = np.sqrt(rr32) > np.sqrt(rp32) * np.float32(1 + 1e-6)
    assert int(nfb.item()) == int(worse.sum())
    # deploy mode with a calibrated tau keeps RMSE within 1% of plain OMP
    tau = lib.calibrate_fallback(rr, rp, 1.01)
    _, _, _, rd, nfd = lib.encode_learned(Dt, Xt, s, net, mode="deploy", tau=tau, sync=True)
    rmse_d = np.sqrt(rd.cpu().numpy().astype(np.float64).mean() / 45)
    rmse_p = np.sqrt(rp_.mean() / 45)
    assert rmse_d <= 1.01 * rmse_p * (1 + 1e-6), (rmse_d, rmse_p)
    tau2 = np.float32(tau) * np.float32(tau)  # FP32, as the kernel compares
    assert int(nfd.item()) == int((rr32 > tau2).sum())
    assert int(nfd.item()) < len(rr32)


def test_trained_network_gains_over_untrained_at_k1024(lib):
    """The learned proposal at the scene's dictionary size: after training on
    (signal, OMP support) pairs, the 2s candidates hold far more of OMP's atoms
    than an untrained network's, and restricted OMP over them comes much closer
    to plain OMP's residual.  Measured at this size: recall about 0.27 against
    0.016, residual RMSE about 1.45x plain OMP's against 2.8x."""
    K, s = 1024, 8
    D = synth.hidden_dictionary(K, 40, rho=0.6)
    Dt = torch.from_numpy(D.astype(np.float32)).cuda()
    Xtr = synth.signals_device(400_000, D, s, 41)
    itr, _, ntr, _ = lib.encode(Dt, Xtr, s, sync=True)
    net = lib.MLP(K, synth.mlp_params(K, 42))
    net.train(Xtr, itr, ntr, epochs=10, batch=8192, lr=1e-2)
    fresh = lib.MLP(K, synth.mlp_params(K, 43))
    Xv = synth.signals_device(20_000, D, s, 44)
    iv, _, nv, rp = lib.encode(Dt, Xv, s, sync=True)
    sup = lib.idx_as_long(iv)
    live = torch.arange(s, device="cuda")[None, :] < nv[:, None].to(torch.int64)

    def scores(n):
        cand = n.propose(Xv, 2 * s)
        c = cand.to(torch.int64) & 0xFFFF
        hit = (sup[:, :, None] == c[:, None, :]).any(dim=2) & live
        _, _, _, rr = lib.encode_restricted(Dt, Xv, cand, s)
        return float(hit.sum()) / float(live.sum()), float((rr.double().sum() / rp.double().sum()).sqrt())

    (r_tr, q_tr), (r_0, q_0) = scores(net), scores(fresh)
    assert r_tr > 0.18 and r_tr > r_0 + 0.15, (r_tr, r_0)
    assert q_tr < 0.75 * q_0, (q_tr, q_0)
