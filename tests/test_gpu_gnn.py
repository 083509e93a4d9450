"""Start-block network on the GPU (bchdav_gnn_*) against its float64 oracle (oracle/gnn.py):
forward output, loss and gradient, Adam trajectory, Ritz-ordered start block."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import device_csr, oracle_csr, to_np
from oracle import gnn

pytestmark = pytest.mark.gpu
D_R, WIDTH = 14, 64


@pytest.fixture(scope="module")
def H():
    import paper_2212_04443_gb300 as P
    return P.Handle()


def _graph(kind):
    if kind == "sbm":
        return synth.sbm_edges(3001, 6, d_in=10, d_out=1.5, seed=41)
    # a hub over the SpMM segment length plus a power-law part
    return synth.disjoint_union(synth.star_edges(2100), synth.rmat_edges(10, seed=42))


def _inputs(H, g, k, seed=0):
    import torch
    A = device_csr(H, g)
    L = oracle_csr(g)
    R = synth.gnn_random_features(g.n, D_R, seed + 1)
    theta = synth.gnn_init(D_R + 2, WIDTH, k, seed=seed + 2)
    return A, L, R, theta, torch.from_numpy(R).cuda(), torch.from_numpy(theta).cuda()


@pytest.mark.parametrize("kind,k", [("sbm", 16), ("hub", 8), ("sbm", 64)])
def test_forward_matches_oracle(H, kind, k):
    g = _graph(kind)
    A, L, R, theta, Rd, Td = _inputs(H, g, k)
    assert H.gnn_n_params(D_R, WIDTH, k) == gnn.n_params(D_R + 2, WIDTH, k) == theta.size
    Z = to_np(H.gnn_forward(A, Rd, Td, WIDTH, k))
    X0 = gnn.features(L, R)
    Zr = gnn.forward(L.scipy(), X0, theta.astype(np.float64), WIDTH, k)[0]
    # float32 through three layers of width 64: relative error a few 1e-6 of the scale
    assert np.abs(Z - Zr).max() <= 1e-4 * np.abs(Zr).max()


@pytest.mark.parametrize("kind,k", [("sbm", 16), ("hub", 8)])
def test_loss_and_gradient_match_oracle(H, kind, k):
    import torch
    g = _graph(kind)
    A, L, R, theta, Rd, Td = _inputs(H, g, k, seed=3)
    w, Y = np.linalg.eigh(L.dense())
    U = np.ascontiguousarray(Y[:, :k])
    loss, grad, Z = H.gnn_loss_grad(A, Rd, Td, torch.from_numpy(U).cuda(), WIDTH, k, ridge=1e-6)
    X0 = gnn.features(L, R)
    lr_, gr_, _ = gnn.loss_and_grad(L.scipy(), X0, theta.astype(np.float64), U, WIDTH, k,
                                    ridge=1e-6)
    assert abs(loss - lr_) <= 1e-4
    grad = to_np(grad)
    # every parameter group agrees to float32 accuracy relative to the group's largest entry
    offs = np.cumsum([0] + [int(np.prod(s)) for s in gnn.param_shapes(D_R + 2, WIDTH, k)])
    for a, b in zip(offs[:-1], offs[1:]):
        scale = max(np.abs(gr_[a:b]).max(), 1e-12)
        assert np.abs(grad[a:b] - gr_[a:b]).max() <= 2e-3 * scale, (a, b)


def test_training_follows_oracle_adam(H):
    """Three Adam steps on two graphs: losses track the float64 oracle's trajectory."""
    import torch
    k, steps, lr = 8, 3, 3e-3
    gs = [synth.sbm_edges(1500, 4, d_in=9, d_out=1, seed=60 + i) for i in range(2)]
    As, Ls, Rs, Rds, Us, Uds = [], [], [], [], [], []
    for i, g in enumerate(gs):
        A = device_csr(H, g)
        L = oracle_csr(g)
        R = synth.gnn_random_features(g.n, D_R, 70 + i)
        U = np.ascontiguousarray(np.linalg.eigh(L.dense())[1][:, :k])
        As.append(A); Ls.append(L); Rs.append(R); Rds.append(torch.from_numpy(R).cuda())
        Us.append(U); Uds.append(torch.from_numpy(U).cuda())
    theta0 = synth.gnn_init(D_R + 2, WIDTH, k, seed=80)
    Td = torch.from_numpy(theta0.copy()).cuda()
    hist = H.gnn_train(As, Rds, Uds, Td, WIDTH, k, steps, lr, ridge=1e-4)
    th = theta0.astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    t = 0
    for s in range(steps):
        for i in range(2):
            loss, grad, _ = gnn.loss_and_grad(Ls[i].scipy(), gnn.features(Ls[i], Rs[i]), th,
                                              Us[i], WIDTH, k, ridge=1e-4)
            assert abs(hist[s, i] - loss) <= 2e-3, (s, i, hist[s, i], loss)
            t += 1
            th, m, v = gnn.adam_step(th, grad, m, v, t, lr)
    assert np.abs(to_np(Td) - th).max() <= 5e-3 * np.abs(th).max()


def test_start_block_is_ritz_ordered(H):
    k = 12
    g = _graph("sbm")
    A, L, R, theta, Rd, Td = _inputs(H, g, k, seed=5)
    V0, ritz = H.gnn_start_block(A, Rd, Td, WIDTH, k)
    V0, ritz = to_np(V0), to_np(ritz)
    assert np.all(np.diff(ritz) >= -1e-14)
    assert np.abs(V0.T @ V0 - np.eye(k)).max() < 1e-12
    S = L.scipy()
    assert np.allclose(np.einsum("ij,ij->j", V0, S @ V0), ritz, atol=1e-12)
    Zr = gnn.forward(S, gnn.features(L, R), theta.astype(np.float64), WIDTH, k)[0]
    _, wr = gnn.start_block(S, Zr)
    # the spans differ by the float32 forward pass only
    assert np.abs(ritz - wr).max() <= 1e-4


FAMILIES = {
    # three training graphs (graph, seed of its solve) and a held-out graph per family
    "rmat": (lambda i: synth.rmat_edges([11, 12, 12][i], seed=300 + i),
             lambda: synth.rmat_edges(13, seed=399), 15),
    "sbm": (lambda i: synth.sbm_edges(30000 + 1000 * i, 16, d_in=16.0, d_out=2.0, seed=700 + i),
            lambda: synth.sbm_edges(60000, 16, d_in=16.0, d_out=2.0, seed=799), 13),
}


@pytest.mark.parametrize("family", ["rmat", "sbm"])
def test_trained_network_on_held_out_graph(H, family):
    """What training buys on an unseen graph of the family.  It learns its graphs and transfers
    (lower alignment loss and lower Ritz values of the start block on the held-out graph), but
    the solve's iteration count does not drop: measured on GB300, R-MAT scale 13 takes 18
    iterations from the trained block and 18 from random blocks; the SBM (60,000 nodes, 16
    clusters) 7 against 6.  The Chebyshev filter of degree 13-15 already brings a random block
    to the wanted subspace within a few iterations, while the network's block (mean Ritz value
    ~0.6 against ~0.1 for the wanted eigenvalues of the SBM) is a poorer start than one filter
    pass.  The test asserts that measured result: no iteration gain over the median of random
    starts."""
    import torch
    import paper_2212_04443_gb300 as P
    train, held, m = FAMILIES[family]
    k, b, act = 16, 8, 48
    As, Rs, Us = [], [], []
    for i in range(3):
        g = train(i)
        A = device_csr(H, g)
        ev, V, info = H.solve(A, k, b, m, act, 1e-8, precision=P.PREC_MIXED, seed=i)
        assert info.status == 0
        for r in range(2):
            As.append(A)
            Us.append(V.contiguous())
            Rs.append(torch.from_numpy(synth.gnn_random_features(g.n, D_R, 400 + 10 * i + r)).cuda())
    g = held()
    At = device_csr(H, g)
    evt, Vt, _ = H.solve(At, k, b, m, act, 1e-8, precision=P.PREC_MIXED, seed=9)
    Rt = torch.from_numpy(synth.gnn_random_features(g.n, D_R, 499)).cuda()
    th0 = torch.from_numpy(synth.gnn_init(D_R + 2, WIDTH, k, seed=11)).cuda()
    theta = th0.clone()
    hist = H.gnn_train(As, Rs, Us, theta, WIDTH, k, 150, 2e-3)
    assert hist[-1].mean() < 0.7 * hist[0].mean()                 # it learns its graphs
    l0 = H.gnn_loss_grad(At, Rt, th0, Vt.contiguous(), WIDTH, k)[0]
    l1 = H.gnn_loss_grad(At, Rt, theta, Vt.contiguous(), WIDTH, k)[0]
    assert l1 < l0                                                # and transfers a little
    V0u, ritz_u = H.gnn_start_block(At, Rt, th0, WIDTH, k)
    V0t, ritz_t = H.gnn_start_block(At, Rt, theta, WIDTH, k)
    assert to_np(ritz_t).mean() < to_np(ritz_u).mean()
    _, _, warm = H.solve(At, k, b, m, act, 1e-8, precision=P.PREC_MIXED, v_init=V0t)
    rnd = [H.solve(At, k, b, m, act, 1e-8, precision=P.PREC_MIXED, seed=s)[2].iters
           for s in range(3)]
    print(f"{family}: held-out alignment loss {l0:.3f} -> {l1:.3f}; mean Ritz value "
          f"{to_np(ritz_u).mean():.3f} -> {to_np(ritz_t).mean():.3f}; iterations warm "
          f"{warm.iters} vs random {rnd}")
    assert warm.status == 0
    # the measured negative result: the trained start block does not save iterations
    assert warm.iters >= int(np.median(rnd))