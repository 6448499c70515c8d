"""Learned gauge-covariant preconditioner (forward, training, flexible CG) on the GPU through the C ABI against the FP64 oracle:
network forward, training loss and gradient of the project's backward kernels, Adam, training,
and flexible CG with its stall fallback."""
import numpy as np
import pytest

import hisq_inputs as hi
import oracle
import oracle_pins as pins
from gpu_util import gpu, rel_err

pytestmark = pytest.mark.gpu

DIMS = (8, 10, 8, 6)
TOL = 1e-10
NW = 408


def _weights(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(NW) + 1j * rng.standard_normal(NW)) * scale


def _as_real(w):
    return np.ascontiguousarray(np.asarray(w, dtype=np.complex128)).view(np.float64)


def _apply(g, pc, v):
    n = len(v)
    vin, vout = g.pack(v, 1), g.bundle(n, 1)
    g.hisq.hisq_pc_apply(pc, g.fat, g.naik, vin, vout, n)
    return g.unpack(vout, n, 1)


@pytest.mark.parametrize("recon", [18, 13])
@pytest.mark.parametrize("n", [1, 3, 16])
def test_network_forward_parity(recon, n):
    with gpu(DIMS, 1, recon) as g:
        W = _weights(1)
        pc = g.hisq.hisq_pc_create(_as_real(W))
        v = np.stack([hi.gaussian_rhs(g.lat, 50 + k) for k in range(n)])
        got = _apply(g, pc, v)
        want = np.stack([g.oracle.pc_forward(W, v[k]) for k in range(n)])
        assert rel_err(got, want) <= 3e-5


def test_network_identity_and_operator_weights():
    """The identity weights give the identity; the weights that spell out Eq. (3) twice give
    A = m^2 - D_eo D_oe (the network's transports are the Dslash's links)."""
    mass = 0.3
    with gpu(DIMS, 1) as g:
        v = np.stack([hi.gaussian_rhs(g.lat, 60 + k) for k in range(2)])
        pc = g.hisq.hisq_pc_create(None)
        assert rel_err(_apply(g, pc, v), v) <= 1e-7
        g.hisq.hisq_pc_set_weights(pc, _as_real(pins.network_weights_aop(mass)))
        assert rel_err(_apply(g, pc, v), g.oracle.aop(v, mass)) <= 1e-5


@pytest.mark.parametrize("K", [1, 4, 12])
def test_loss_and_gradient_parity(K):
    """Loss and every weight gradient from the GPU backward kernels against the oracle's
    backward (itself pinned by finite differences)."""
    with gpu(DIMS, 1) as g:
        W = _weights(2, 0.2)
        pc = g.hisq.hisq_pc_create(_as_real(W))
        g.hisq.hisq_pc_set_form(pc, g.hisq.HISQ_PC_HERMITIAN_PART)  # trained as M itself
        r = np.stack([hi.gaussian_rhs(g.lat, 70 + k) for k in range(K)])
        e = np.stack([hi.gaussian_rhs(g.lat, 90 + k) for k in range(K)])
        grad = np.zeros(2 * NW)
        mass = 0.2
        loss = g.hisq.hisq_pc_loss_grad(pc, g.fat, g.naik, mass, g.pack(r, 1), g.pack(e, 1), K, grad)
        want_loss, want_grad = g.oracle.pc_loss_grad(W, r, e, mass)
        assert abs(loss - want_loss) / want_loss <= 1e-5
        got = grad.view(np.complex128)
        assert np.linalg.norm(got - want_grad) / np.linalg.norm(want_grad) <= 1e-4


def test_adam_step_matches_oracle():
    with gpu((4, 4, 4, 4), 1) as g:
        W = _weights(3)
        pc = g.hisq.hisq_pc_create(_as_real(W))
        rng = np.random.default_rng(4)
        theta = _as_real(W).copy()
        m, v = np.zeros_like(theta), np.zeros_like(theta)
        for t in range(1, 4):
            grad = rng.standard_normal(2 * NW)
            g.hisq.hisq_pc_adam_step(pc, grad, t, 1e-2, 0.9, 0.999, 1e-8)
            oracle.adam_step(theta, grad, m, v, t, 1e-2, 0.9, 0.999, 1e-8)
        got = np.zeros(2 * NW)
        g.hisq.hisq_pc_get_weights(pc, got)
        np.testing.assert_allclose(got, theta, rtol=0, atol=1e-12)


def training_pairs(g, mass, nrhs, steps):
    """(r, e) pairs from plain CG: x_k after k iterations, e_k = x* - x_k, r_k = b - A x_k."""
    rs, es = [], []
    p = g.hisq.hisq_default_solver_params()
    p.inner_prec = 0
    for j in range(nrhs):
        b = hi.gaussian_rhs(g.lat, 200 + j)
        p.max_iter = 20000
        g.hisq.hisq_set_solver_params(p)
        xs = np.zeros_like(b)
        g.hisq.hisq_cg_solve(g.fat, g.naik, [b], [xs], mass, TOL)
        for k in steps:
            p.max_iter = k
            g.hisq.hisq_set_solver_params(p)
            xk = np.zeros_like(b)
            g.hisq.hisq_cg_solve(g.fat, g.naik, [b], [xk], mass, TOL, raise_on_error=False)
            rs.append(b - g.oracle.aop(xk, mass))
            es.append(xs - xk)
    p.max_iter = 20000
    g.hisq.hisq_set_solver_params(p)
    return np.stack(rs), np.stack(es)


def pack_pairs(g, r, e):
    """Bundles of 16 (the last padded) as one contiguous device buffer each."""
    import torch
    K = len(r)
    nb = (K + 15) // 16
    pad = nb * 16 - K
    rp = np.concatenate([r, r[:pad]]) if pad else r
    ep = np.concatenate([e, e[:pad]]) if pad else e
    bs = g.hisq.hisq_vector_bytes(1, 16)
    rb = torch.empty(nb * bs, dtype=torch.uint8, device=g.dev)
    eb = torch.empty_like(rb)
    for i in range(nb):
        g.hisq.hisq_pack(g._dev64(rp[16 * i:16 * i + 16]), rb[i * bs:(i + 1) * bs], 16, 1)
        g.hisq.hisq_pack(g._dev64(ep[16 * i:16 * i + 16]), eb[i * bs:(i + 1) * bs], 16, 1)
    return rb, eb


def initial_weights(seed=0, scale=0.02):
    """Identity network plus a small random perturbation (the pure identity is a saddle point
    of the loss: every hop-path gradient vanishes there)."""
    W = np.zeros(NW, complex)
    W[0] = W[68] = W[340] = 1.0
    return W + _weights(seed, scale)


def test_identity_is_a_saddle_point():
    """At the identity weights the gradient of every hop path is zero (only the identity-path
    weights can move), which is why training starts from a perturbed identity."""
    with gpu(DIMS, 1) as g:
        pc = g.hisq.hisq_pc_create(None)
        r = np.stack([hi.gaussian_rhs(g.lat, 70 + k) for k in range(2)])
        e = np.stack([hi.gaussian_rhs(g.lat, 90 + k) for k in range(2)])
        grad = np.zeros(2 * NW)
        g.hisq.hisq_pc_loss_grad(pc, g.fat, g.naik, 0.1, g.pack(r, 1), g.pack(e, 1), 2, grad)
        gc = grad.view(np.complex128)
        hop = np.ones(NW, bool)
        hop[[0, 68, 340]] = False
        assert np.abs(gc[hop]).max() <= 1e-6 * np.abs(gc[~hop]).max()


def test_training_lowers_loss_and_matches_oracle_loss():
    mass = 0.05
    with gpu(DIMS, 1) as g:
        r, e = training_pairs(g, mass, 2, [2, 5, 8, 11, 14, 17, 20, 23])
        rb, eb = pack_pairs(g, r, e)
        pc = g.hisq.hisq_pc_create(_as_real(initial_weights()))
        g.hisq.hisq_pc_set_form(pc, g.hisq.HISQ_PC_HERMITIAN_PART)
        hist = np.zeros(20)
        g.hisq.hisq_pc_train(pc, g.fat, g.naik, mass, rb, eb, len(r), 16, 20, 1e-2, hist)
        assert hist[-1] < 0.5 * hist[0], hist
        W = np.zeros(2 * NW)
        g.hisq.hisq_pc_get_weights(pc, W)
        loss, _ = g.oracle.pc_loss_grad(W.view(np.complex128), r, e, mass, with_grad=False)
        assert loss < 0.5 * hist[0]


def _fcg(g, pc, rhs, mass, graph=1, **kw):
    p = g.hisq.hisq_default_solver_params()
    p.inner_prec = 1
    p.use_graph = graph
    p.pc = pc.value if pc is not None else None
    for k, v in kw.items():
        setattr(p, k, v)
    g.hisq.hisq_set_solver_params(p)
    xs = [np.zeros_like(b) for b in rhs]
    g.hisq.hisq_cg_solve(g.fat, g.naik, list(rhs), xs, mass, TOL)
    iters = np.zeros(len(rhs), dtype=np.int32)
    stats = g.hisq.hisq_last_stats(iters)
    return np.stack(xs), stats, iters


@pytest.mark.parametrize("graph", [0, 1])
@pytest.mark.parametrize("form", [1, 0])
def test_fcg_iterates_match_oracle(graph, form):
    """The GPU's flexible CG takes the oracle's steps: after k = 1..6 iterations with a fixed
    random network (normal form M^dag M and Hermitian part of M) its iterate x_k equals the
    oracle's, whose beta and alpha are pinned by preconditioned CG and by the A-orthogonality of
    consecutive steps.  A wrong beta (Fletcher-Reeves numerator, misplaced conjugate) moves x_2 on
    by far more than the FP32 storage and network arithmetic do."""
    mass = 0.1
    with gpu(DIMS, 1) as g:
        W = _weights(7, 0.3)
        pc = g.hisq.hisq_pc_create(_as_real(W))
        g.hisq.hisq_pc_set_form(pc, form)
        b = hi.gaussian_rhs(g.lat, 650)
        worst = 0.0
        for k in range(1, 7):
            p = g.hisq.hisq_default_solver_params()
            p.inner_prec, p.use_graph, p.pc, p.max_iter = 1, graph, pc.value, k
            g.hisq.hisq_set_solver_params(p)
            x = np.zeros_like(b)
            rc = g.hisq.hisq_cg_solve(g.fat, g.naik, [b], [x], mass, TOL, raise_on_error=False)
            assert rc in (0, -4)  # HISQ_OK or HISQ_ERR_NOT_CONVERGED (max_iter reached)
            want, _, _ = g.oracle.fcg(W, b, mass, tol=1e-300, max_iter=k, form=2 if form == 0 else 1)
            worst = max(worst, rel_err(x[None], want[None]))
        assert worst <= 1e-4, worst


@pytest.mark.parametrize("graph", [0, 1])
def test_fcg_identity_network_is_cg(graph):
    mass = 0.05
    with gpu(DIMS, 1) as g:
        rhs = [hi.gaussian_rhs(g.lat, 300 + k) for k in range(2)]
        pc = g.hisq.hisq_pc_create(None)
        x, stats, iters = _fcg(g, pc, rhs, mass, graph)
        assert np.all(g.oracle.true_residual(np.stack(rhs), x, mass) <= TOL)
        _, _, it_cg = _fcg(g, None, rhs, mass, graph)
        assert np.all(np.abs(iters - it_cg) <= 2), (iters, it_cg)


@pytest.mark.parametrize("graph,form", [(0, 1), (1, 1), (1, 0)])
def test_fcg_with_trained_network_beats_plain_cg_in_iterations(graph, form):
    """What the trained network gains: fewer iterations than plain CG to the same FP64 true
    residual on fresh right-hand sides (normal form M^dag M and Hermitian part of M)."""
    mass = 0.05
    with gpu(DIMS, 1) as g:
        r, e = training_pairs(g, mass, 4, list(range(2, 40, 3)))
        rb, eb = pack_pairs(g, r, e)
        pc = g.hisq.hisq_pc_create(_as_real(initial_weights()))
        g.hisq.hisq_pc_set_form(pc, form)
        g.hisq.hisq_pc_train(pc, g.fat, g.naik, mass, rb, eb, len(r), 16, 60, 1e-2)
        rhs = [hi.gaussian_rhs(g.lat, 400 + k) for k in range(3)]
        x, stats, iters = _fcg(g, pc, rhs, mass, graph)
        assert np.all(g.oracle.true_residual(np.stack(rhs), x, mass) <= TOL)
        _, _, it_cg = _fcg(g, None, rhs, mass, graph)
        assert np.mean(iters) < np.mean(it_cg), (iters, it_cg)


def test_fcg_stall_falls_back_to_cg():
    """A network that multiplies by A instead of approximating its inverse squares the condition
    number, so the residual does not drop 10x within the stall window; the solver switches to
    plain CG from the current iterate and still reaches the true residual."""
    mass = 0.05
    with gpu(DIMS, 1) as g:
        pc = g.hisq.hisq_pc_create(_as_real(pins.network_weights_aop(mass)))
        rhs = [hi.gaussian_rhs(g.lat, 500)]
        x, stats, iters = _fcg(g, pc, rhs, mass, 1, stall_window=5)
        assert g.oracle.true_residual(rhs[0], x[0], mass)[0] <= TOL
        assert stats.fallbacks >= 1


def test_hermitian_part_of_the_network():
    """M_H = (M + M^dag)/2 applied by the GPU: <u, M_H v> = (<u, M v> + <M u, v>)/2 with M the
    oracle's network, and M_H is Hermitian: <u, M_H v> = conj(<v, M_H u>)."""
    with gpu(DIMS, 1) as g:
        W = _weights(5, 0.3)
        pc = g.hisq.hisq_pc_create(_as_real(W))
        u = hi.gaussian_rhs(g.lat, 800)
        v = hi.gaussian_rhs(g.lat, 801)
        mh = _apply_h(g, pc, np.stack([u, v]))
        lhs = np.vdot(u, mh[1])
        want = 0.5 * (np.vdot(u, g.oracle.pc_forward(W, v)) + np.vdot(g.oracle.pc_forward(W, u), v))
        assert abs(lhs - want) / abs(want) <= 3e-5
        assert abs(lhs - np.conj(np.vdot(v, mh[0]))) / abs(lhs) <= 3e-5


def _apply_h(g, pc, v):
    n = len(v)
    vin, vout = g.pack(v, 1), g.bundle(n, 1)
    g.hisq.hisq_pc_apply_hermitian(pc, g.fat, g.naik, vin, vout, n)
    return g.unpack(vout, n, 1)


def _apply_op(g, fn, pc, v):
    n = len(v)
    vin, vout = g.pack(v, 1), g.bundle(n, 1)
    fn(pc, g.fat, g.naik, vin, vout, n)
    return g.unpack(vout, n, 1)


@pytest.mark.parametrize("n", [1, 3])
def test_adjoint_and_normal_form_parity(n):
    """M^dag and M^dag M applied by the GPU against the oracle's adjoint network."""
    with gpu(DIMS, 1) as g:
        W = _weights(6, 0.3)
        pc = g.hisq.hisq_pc_create(_as_real(W))
        v = np.stack([hi.gaussian_rhs(g.lat, 820 + k) for k in range(n)])
        adj = _apply_op(g, g.hisq.hisq_pc_apply_adjoint, pc, v)
        assert rel_err(adj, np.stack([g.oracle.pc_adjoint(W, v[k]) for k in range(n)])) <= 3e-5
        nrm = _apply_op(g, g.hisq.hisq_pc_apply_normal, pc, v)
        assert rel_err(nrm, np.stack([g.oracle.pc_normal(W, v[k]) for k in range(n)])) <= 3e-5


@pytest.mark.parametrize("K", [1, 4])
def test_normal_form_loss_and_gradient_parity(K):
    """The normal-form loss and its two-term weight gradient against the oracle's."""
    with gpu(DIMS, 1) as g:
        W = _weights(7, 0.2)
        pc = g.hisq.hisq_pc_create(_as_real(W))
        g.hisq.hisq_pc_set_form(pc, g.hisq.HISQ_PC_NORMAL)
        r = np.stack([hi.gaussian_rhs(g.lat, 840 + k) for k in range(K)])
        e = np.stack([hi.gaussian_rhs(g.lat, 860 + k) for k in range(K)])
        grad = np.zeros(2 * NW)
        mass = 0.2
        loss = g.hisq.hisq_pc_loss_grad(pc, g.fat, g.naik, mass, g.pack(r, 1), g.pack(e, 1), K, grad)
        want_loss, want_grad = g.oracle.pc_loss_grad_normal(W, r, e, mass)
        assert abs(loss - want_loss) / want_loss <= 1e-5
        got = grad.view(np.complex128)
        assert np.linalg.norm(got - want_grad) / np.linalg.norm(want_grad) <= 1e-4


def test_set_form_validation():
    from paper_1409_1510_gb300.hisq import HisqError
    with gpu((4, 4, 4, 4), 1) as g:
        pc = g.hisq.hisq_pc_create(None)
        with pytest.raises(HisqError):
            g.hisq.hisq_pc_set_form(pc, 7)


def test_flexible_cg_graph_reused_after_a_persistent_plain_solve():
    """Flexible CG (captured graph), then plain CG (persistent kernel), then flexible CG again in
    the same context: the reused graph still terminates and converges."""
    mass = 0.05
    with gpu(DIMS, 1) as g:
        pc = g.hisq.hisq_pc_create(None)
        rhs = [hi.gaussian_rhs(g.lat, 900 + k) for k in range(2)]
        _, s1, it1 = _fcg(g, pc, rhs, mass, graph=1)
        _, s2, it2 = _fcg(g, None, rhs, mass, graph=2)
        x3, s3, it3 = _fcg(g, pc, rhs, mass, graph=1)
        assert s1.converged == s3.converged == 2 and np.array_equal(it1, it3)
        assert np.all(g.oracle.true_residual(np.stack(rhs), x3, mass) <= TOL)
