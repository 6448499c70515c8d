"""Checks that tie the FP64 oracle to facts fixed by the paper and by mathematics, not to itself.

Each ``pin_*`` function takes an ``oracle.Oracle`` factory and returns a (passed, detail) pair, so
that the same checks serve the pin tests (which assert them) and the mutation test (which plants
a mistake in a copy of the oracle and expects at least one pin to fail).
"""
import numpy as np

import hisq_inputs as hi
import oracle.dense as dense


def _rand_vec(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _fields(dims, seed_shift=0):
    lat = hi.Lattice(dims)
    return lat, hi.fat_links(lat, seed_u=1 + seed_shift, seed_noise=2 + seed_shift), \
        hi.naik_links(lat, seed_u=3 + seed_shift)


def pin_matrix_form(make, dims=(4, 4, 4, 4), tol=1e-13):
    """Stencil oracle equals the sparse matrix assembled block by block from Eq. (3), on the full
    lattice and for both even-odd blocks."""
    lat, X, N = _fields(dims)
    o = make(dims, X, N)
    rng = np.random.default_rng(11)
    D = dense.dslash_matrix(dims, X, N)
    v = _rand_vec(rng, (2, lat.volume, 3))
    worst = 0.0
    w = o.dslash_full(v)
    for k in range(2):
        worst = max(worst, _rel(w[k].ravel(), D @ v[k].ravel()))
    deo, doe = dense.even_odd_blocks(dims, X, N)
    ve = _rand_vec(rng, (lat.half_volume, 3))
    worst = max(worst, _rel(o.dslash_eo(ve, 1).ravel(), doe @ ve.ravel()))
    worst = max(worst, _rel(o.dslash_eo(ve, 0).ravel(), deo @ ve.ravel()))
    return worst <= tol, f"max rel diff {worst:.3e} on {dims}"


def pin_anti_hermitian(make, dims=(8, 4, 6, 4), tol=1e-14):
    """<u, D_eo v> = -<D_oe u, v> and <u, D v> = -<D u, v> (D is anti-Hermitian for any links)."""
    lat, X, N = _fields(dims)
    o = make(dims, X, N)
    rng = np.random.default_rng(12)
    u = _rand_vec(rng, (lat.half_volume, 3))
    v = _rand_vec(rng, (lat.half_volume, 3))
    lhs = np.vdot(u, o.dslash_eo(v, 0))
    rhs = -np.vdot(o.dslash_eo(u, 1), v)
    err1 = abs(lhs - rhs) / abs(lhs)
    uf = _rand_vec(rng, (lat.volume, 3))
    vf = _rand_vec(rng, (lat.volume, 3))
    a = np.vdot(uf, o.dslash_full(vf))
    b = -np.vdot(o.dslash_full(uf), vf)
    err2 = abs(a - b) / abs(a)
    return max(err1, err2) <= tol, f"eo {err1:.2e} full {err2:.2e}"


def gauge_transform(lat, X, N, omega):
    """X'_{x,mu} = W_x X_{x,mu} W^dag_{x+mu}, N'_{x,mu} = W_x N_{x,mu} W^dag_{x+3mu}."""
    c = lat.coords()
    Xp = np.empty_like(X)
    Np = np.empty_like(N)
    for mu in range(4):
        for step, src, dst in ((1, X, Xp), (3, N, Np)):
            cc = c.copy()
            cc[:, mu] = (cc[:, mu] + step) % lat.dims[mu]
            lx, ly, lz, _ = lat.dims
            nb = cc[:, 0] + lx * (cc[:, 1] + ly * (cc[:, 2] + lz * cc[:, 3]))
            dst[mu] = omega @ src[mu] @ omega[nb].conj().swapaxes(-1, -2)
    return Xp, Np


def pin_gauge_covariance(make, dims=(8, 4, 4, 6), tol=1e-13):
    """D' (W v) = W (D v) for a random SU(3) gauge transform W, full lattice and even-odd."""
    lat, X, N = _fields(dims)
    om = hi.gauge_transform_field(lat)
    Xp, Np = gauge_transform(lat, X, N, om)
    o, op = make(dims, X, N), make(dims, Xp, Np)
    rng = np.random.default_rng(13)
    v = _rand_vec(rng, (lat.volume, 3))
    lhs = op.dslash_full(np.einsum("xab,xb->xa", om, v))
    rhs = np.einsum("xab,xb->xa", om, o.dslash_full(v))
    err = _rel(lhs, rhs)
    ve = _rand_vec(rng, (lat.half_volume, 3))
    ev, od = lat.eo_sites(0), lat.eo_sites(1)
    lhs = op.dslash_eo(np.einsum("xab,xb->xa", om[ev], ve), 1)
    rhs = np.einsum("xab,xb->xa", om[od], o.dslash_eo(ve, 1))
    err = max(err, _rel(lhs, rhs))
    return err <= tol, f"rel {err:.2e}"


def free_field_eigenvalue(dims, k, mass, c1, c3, antiperiodic_t=True):
    """Closed form: A = m^2 - D_eo D_oe on the plane wave exp(i p.x) restricted to even sites has
    eigenvalue m^2 + 4 sum_mu (c1 sin p_mu + c3 sin 3 p_mu)^2, p_mu = 2 pi k_mu / L_mu
    (k_t + 1/2 for the antiperiodic t direction).  Follows from D^2 = sum_mu S_mu^2 for unit
    links, because the staggered phases anticommute between directions."""
    p = [2 * np.pi * (k[mu] + (0.5 if (mu == 3 and antiperiodic_t) else 0.0)) / dims[mu] for mu in range(4)]
    return mass ** 2 + 4 * sum((c1 * np.sin(q) + c3 * np.sin(3 * q)) ** 2 for q in p), p


def plane_wave_even(lat, p, colour):
    c = lat.coords()[lat.eo_sites(0)]
    f = np.zeros((lat.half_volume, 3), dtype=np.complex128)
    f[:, colour] = np.exp(1j * (c @ np.asarray(p)))
    return f


def pin_free_field_plane_waves(make, dims=(8, 8, 6, 10), mass=0.3, tol=1e-13, n_modes=12):
    """A applied to even-site plane waves of the unit-link field returns the closed-form
    eigenvalue times the wave (checks directions, hop lengths 1 and 3, signs, coefficients and
    the antiperiodic boundary)."""
    lat = hi.Lattice(dims)
    c1, c3 = 9.0 / 8.0, -1.0 / 24.0
    X, N = hi.free_field_links(lat, c1, c3)
    o = make(dims, X, N)
    rng = np.random.default_rng(14)
    worst = 0.0
    for _ in range(n_modes):
        k = [int(rng.integers(0, d)) for d in dims]
        lam, p = free_field_eigenvalue(dims, k, mass, c1, c3)
        f = plane_wave_even(lat, p, int(rng.integers(0, 3)))
        worst = max(worst, _rel(o.aop(f, mass), lam * f))
    return worst <= tol, f"max rel {worst:.2e}"


def pin_free_field_spectrum(make, dims=(4, 4, 4, 6), mass=0.2, tol=1e-11):
    """Sorted eigenvalues of the matrix of A (built column by column from the oracle) equal the
    closed-form free-field spectrum with multiplicities."""
    lat = hi.Lattice(dims)
    c1, c3 = 9.0 / 8.0, -1.0 / 24.0
    X, N = hi.free_field_links(lat, c1, c3)
    o = make(dims, X, N)
    n = lat.half_volume * 3
    eye = np.eye(n, dtype=np.complex128).reshape(n, lat.half_volume, 3)
    A = o.aop(eye, mass).reshape(n, n).T
    got = np.sort(np.linalg.eigvalsh(0.5 * (A + A.conj().T)))
    vals = []
    for kx in range(dims[0]):
        for ky in range(dims[1]):
            for kz in range(dims[2]):
                for kt in range(dims[3]):
                    vals += [free_field_eigenvalue(dims, (kx, ky, kz, kt), mass, c1, c3)[0]] * 3
    want = np.sort(vals)[::2]  # p and p + (pi,pi,pi,pi) coincide on even sites
    herm = _rel(A, A.conj().T)
    err = float(np.max(np.abs(got - want)) / np.max(want))
    return err <= tol and herm <= 1e-14, f"spectrum {err:.2e}, hermiticity {herm:.2e}"


def pin_cg_dense_solve(make, dims=(4, 4, 4, 6), mass=0.1, tol=1e-10):
    """Oracle CG meets the true residual and agrees with a dense direct solve of the matrix A
    assembled from Eq. (3)."""
    lat, X, N = _fields(dims)
    o = make(dims, X, N)
    b = hi.gaussian_rhs(lat, 0)
    x, it, rel = o.cg(b, mass, tol=tol)
    A = dense.a_matrix(dims, X, N, mass).toarray()
    xd = np.linalg.solve(A, b.ravel())
    ev = np.linalg.eigvalsh(A)
    kappa = ev[-1] / ev[0]
    err = _rel(x.ravel(), xd)
    true = np.linalg.norm(b.ravel() - A @ x.ravel()) / np.linalg.norm(b)
    ok = it > 0 and rel <= tol and true <= tol * 1.01 and err <= kappa * tol and it <= A.shape[0]
    return ok, f"iters {it}, true {true:.2e}, |x-xd|/|xd| {err:.2e}, kappa {kappa:.1f}"


def pin_cg_free_field_exact(make, dims=(8, 8, 8, 8), mass=0.05, tol=1e-10):
    """CG on the unit-link field reproduces the momentum-space solution x = sum c_p f_p / lambda_p
    for a right-hand side made of a few plane waves."""
    lat = hi.Lattice(dims)
    c1, c3 = 9.0 / 8.0, -1.0 / 24.0
    X, N = hi.free_field_links(lat, c1, c3)
    o = make(dims, X, N)
    rng = np.random.default_rng(15)
    b = np.zeros((lat.half_volume, 3), dtype=np.complex128)
    x_exact = np.zeros_like(b)
    for _ in range(5):
        k = [int(rng.integers(0, d)) for d in dims]
        lam, p = free_field_eigenvalue(dims, k, mass, c1, c3)
        coef = complex(rng.standard_normal(), rng.standard_normal())
        f = plane_wave_even(lat, p, int(rng.integers(0, 3)))
        b += coef * f
        x_exact += coef * f / lam
    x, it, rel = o.cg(b, mass, tol=tol)
    err = _rel(x, x_exact)
    return it > 0 and err <= 1e-8, f"iters {it}, rel err {err:.2e}"


MULTISHIFTS = (0.003, 0.0, 0.05, -0.004, 1.0)


def pin_multishift_dense_solve(make, dims=(4, 4, 4, 6), mass=0.1, tol=1e-10, shifts=MULTISHIFTS):
    """Multi-shift CG: every x_j agrees with a dense direct solve of A + sigma_j (A assembled from
    Eq. (3)), within its condition number times tol, and meets the true residual; the shifts are
    unsorted and one is negative (sigma > -m^2), so the base system is not the first one."""
    lat, X, N = _fields(dims)
    o = make(dims, X, N)
    b = hi.gaussian_rhs(lat, 1)
    xs, it, its, rels = o.cg_multishift(b, shifts, mass, tol=tol, max_iter=2000)
    A = dense.a_matrix(dims, X, N, mass).toarray()
    ev = np.linalg.eigvalsh(A)
    worst, detail = 0.0, []
    ok = it > 0
    for j, s in enumerate(shifts):
        As = A + s * np.eye(A.shape[0])
        xd = np.linalg.solve(As, b.ravel())
        kappa = (ev[-1] + s) / (ev[0] + s)
        err = _rel(xs[j].ravel(), xd)
        true = np.linalg.norm(b.ravel() - As @ xs[j].ravel()) / np.linalg.norm(b)
        ok &= its[j] > 0 and true <= tol * 1.01 and rels[j] <= tol and err <= kappa * tol
        worst = max(worst, err / (kappa * tol))
        detail.append(its[j])
    # the base (smallest shift) is the slowest system: it stops last
    ok &= its[int(np.argmin(shifts))] == it
    return bool(ok), f"base iters {it}, per shift {detail}, worst err/(kappa tol) {worst:.2f}"


def pin_multishift_free_field_exact(make, dims=(8, 8, 8, 8), mass=0.05, tol=1e-10, shifts=(0.0, 0.02, 0.3, 2.0)):
    """Multi-shift CG on the unit-link field reproduces x_j = sum c_p f_p / (lambda_p + sigma_j)
    for a right-hand side made of a few plane waves (closed-form eigenvalues)."""
    lat = hi.Lattice(dims)
    c1, c3 = 9.0 / 8.0, -1.0 / 24.0
    X, N = hi.free_field_links(lat, c1, c3)
    o = make(dims, X, N)
    rng = np.random.default_rng(16)
    b = np.zeros((lat.half_volume, 3), dtype=np.complex128)
    x_exact = np.zeros((len(shifts), lat.half_volume, 3), dtype=np.complex128)
    for _ in range(6):
        k = [int(rng.integers(0, d)) for d in dims]
        lam, p = free_field_eigenvalue(dims, k, mass, c1, c3)
        coef = complex(rng.standard_normal(), rng.standard_normal())
        f = plane_wave_even(lat, p, int(rng.integers(0, 3)))
        b += coef * f
        for j, s in enumerate(shifts):
            x_exact[j] += coef * f / (lam + s)
    xs, it, its, rels = o.cg_multishift(b, shifts, mass, tol=tol, max_iter=2000)
    errs = [_rel(xs[j], x_exact[j]) for j in range(len(shifts))]
    return it > 0 and max(errs) <= 1e-8, f"iters {it} {list(its)}, rel errs {max(errs):.2e}"


def pin_trace_z2_unbiased(make, dims=(4, 4, 4, 6), mass=0.2, nnoise=96, seed=11, tol=1e-10):
    """Eq. (2) without derivative factors: the Z2-noise estimate of Tr A^{-1} lies within four
    standard errors of the exact trace of the dense inverse, where the error is the exact
    standard deviation of a real-Z2 estimate of a Hermitian B = A^{-1},
    sqrt(2 sum_{i != j} (Re B_ij)^2 / N); and its noise is +-1 with both signs present."""
    lat, X, N = _fields(dims)
    o = make(dims, X, N)
    mean, samples = o.trace_inverse(mass, nnoise, seed, tol)
    B = np.linalg.inv(dense.a_matrix(dims, X, N, mass).toarray())
    exact = float(np.trace(B).real)
    off = B.real - np.diag(np.diag(B.real))
    sigma = float(np.sqrt(2.0 * np.sum(off ** 2) / nnoise))
    ok = np.isfinite(mean) and abs(mean - exact) <= 4.0 * sigma
    return bool(ok), f"estimate {mean:.6f} exact {exact:.6f} sigma {sigma:.2e}"


def pin_condensate_identity(make, dims=(4, 4, 4, 6), mass=0.3):
    """Tr M^{-1} of the staggered matrix M = m + D (D assembled from Eq. (3), both parities)
    equals 2 m Tr A^{-1} (A from the oracle, column by column); this ties the even-site trace the
    estimator targets to the full fermion matrix."""
    lat, X, N = _fields(dims)
    o = make(dims, X, N)
    n = lat.half_volume * 3
    eye = np.eye(n, dtype=np.complex128).reshape(n, lat.half_volume, 3)
    A = o.aop(eye, mass).reshape(n, n).T
    D = dense.dslash_matrix(dims, X, N).toarray()
    M = mass * np.eye(D.shape[0]) + D
    full = np.trace(np.linalg.inv(M))
    half = 2.0 * mass * np.trace(np.linalg.inv(A))
    err = abs(full - half) / abs(full)
    return err <= 1e-11, f"Tr M^-1 {full:.8f}, 2 m Tr A^-1 {half:.8f}, rel {err:.1e}"


def network_weights_identity():
    """Weights with only the identity path of channel 0 set: the network is the identity."""
    W1 = np.zeros((17, 4, 1), complex); W1[0, 0, 0] = 1
    W2 = np.zeros((17, 4, 4), complex); W2[0, 0, 0] = 1
    W3 = np.zeros((17, 1, 4), complex); W3[0, 0, 0] = 1
    return np.concatenate([W1.ravel(), W2.ravel(), W3.ravel()])


def network_weights_aop(mass):
    """Weights for which the network computes A r = m^2 r - D_eo D_oe r: channel 0 carries
    D(D r) through the hop paths (+1 on forward, -1 on backward hops reproduces Eq. (3)),
    channel 1 carries r through the identity path."""
    hop = np.zeros(17, complex)
    for mu in range(4):
        hop[1 + 2 * mu], hop[2 + 2 * mu] = 1, -1
        hop[9 + 2 * mu], hop[10 + 2 * mu] = 1, -1
    W1 = np.zeros((17, 4, 1), complex); W1[:, 0, 0] = hop; W1[0, 1, 0] = 1
    W2 = np.zeros((17, 4, 4), complex); W2[:, 0, 0] = hop; W2[0, 1, 1] = 1
    W3 = np.zeros((17, 1, 4), complex); W3[0, 0, 0] = -1; W3[0, 0, 1] = mass ** 2
    return np.concatenate([W1.ravel(), W2.ravel(), W3.ravel()])


def pin_network_loss_zero_at_inverse(make, dims=(4, 4, 4, 4), mass=0.4, tol=1e-12):
    """The loss vanishes for pairs the network maps exactly: with the weights that spell out A,
    the pairs (r, e) = (v, A v) give M r = e, so loss = 0; scaling e by 1/2 gives exactly
    |A (A v / 2)|^2 / |v|^2 per pair (a closed form of the residual-norm loss)."""
    lat, X, N = _fields(dims)
    o = make(dims, X, N)
    W = network_weights_aop(mass)
    v = np.stack([hi.gaussian_rhs(lat, 30 + k) for k in range(2)])
    Av = o.aop(v, mass)
    l0, _ = o.pc_loss_grad(W, v, Av, mass, False)
    l1, _ = o.pc_loss_grad(W, v, 0.5 * Av, mass, False)
    AAv = o.aop(0.5 * Av, mass)
    want = np.mean([np.vdot(AAv[k], AAv[k]).real / np.vdot(v[k], v[k]).real for k in range(2)])
    return l0 <= tol and abs(l1 - want) <= 1e-12 * want, f"zero {l0:.1e}, closed form {abs(l1 - want) / want:.1e}"


def pin_network_special_weights(make, dims=(8, 4, 4, 6), mass=0.2, tol=1e-13):
    """Identity weights give the identity; the weights that spell out Eq. (3) twice give A."""
    lat, X, N = _fields(dims)
    o = make(dims, X, N)
    r = hi.gaussian_rhs(lat, 3)
    e1 = _rel(o.pc_forward(network_weights_identity(), r), r)
    e2 = _rel(o.pc_forward(network_weights_aop(mass), r), o.aop(r, mass))
    return max(e1, e2) <= tol, f"identity {e1:.1e}, A {e2:.1e}"


def pin_network_covariance(make, dims=(6, 4, 4, 8), tol=1e-13):
    """The network commutes with gauge transforms: M'(W r) = W (M r)."""
    lat, X, N = _fields(dims)
    om = hi.gauge_transform_field(lat)
    Xp, Np = gauge_transform(lat, X, N, om)
    o, op = make(dims, X, N), make(dims, Xp, Np)
    rng = np.random.default_rng(16)
    W = _rand_vec(rng, o.pc_num_weights) * 0.3
    r = hi.gaussian_rhs(lat, 4)
    ev = lat.eo_sites(0)
    lhs = op.pc_forward(W, np.einsum("xab,xb->xa", om[ev], r))
    rhs = np.einsum("xab,xb->xa", om[ev], o.pc_forward(W, r))
    err = _rel(lhs, rhs)
    return err <= tol, f"rel {err:.2e}"


def pin_network_gradient_fd(make, dims=(4, 4, 4, 4), n_checks=24, tol=1e-6):
    """Analytic loss gradient equals central finite differences in Re W and Im W."""
    lat, X, N = _fields(dims)
    o = make(dims, X, N)
    rng = np.random.default_rng(17)
    W = _rand_vec(rng, o.pc_num_weights) * 0.3
    r = np.stack([hi.gaussian_rhs(lat, 10 + k) for k in range(2)])
    e = np.stack([hi.gaussian_rhs(lat, 20 + k) for k in range(2)])
    mass = 0.3
    _, g = o.pc_loss_grad(W, r, e, mass)
    h = 1e-5
    worst = 0.0
    for i in rng.choice(W.size, n_checks, replace=False):
        for unit, comp in ((1.0, g[i].real), (1j, g[i].imag)):
            Wp, Wm = W.copy(), W.copy()
            Wp[i] += unit * h
            Wm[i] -= unit * h
            fd = (o.pc_loss_grad(Wp, r, e, mass, False)[0] - o.pc_loss_grad(Wm, r, e, mass, False)[0]) / (2 * h)
            worst = max(worst, abs(fd - comp) / max(abs(comp), 1e-3 * np.abs(g).max()))
    return worst <= tol, f"worst rel {worst:.2e}"


def pin_fcg_identity_is_cg(make, dims=(4, 4, 4, 6), mass=0.1, tol=1e-10):
    """Flexible CG with the identity network takes the same iterations as CG and reaches the
    dense-solve solution."""
    lat, X, N = _fields(dims)
    o = make(dims, X, N)
    b = hi.gaussian_rhs(lat, 5)
    x1, it1, _ = o.cg(b, mass, tol=tol)
    x2, it2, rel2 = o.fcg(network_weights_identity(), b, mass, tol=tol)
    A = dense.a_matrix(dims, X, N, mass).toarray()
    xd = np.linalg.solve(A, b.ravel())
    err = _rel(x2.ravel(), xd)
    return abs(it1 - it2) <= 1 and rel2 <= tol and err <= 1e-7, f"cg {it1} fcg {it2} err {err:.1e}"


def pin_network_adjoint(make, dims=(6, 4, 4, 4), tol=1e-13):
    """The adjoint network is the adjoint of the forward one: <u, M v> = <M^dag u, v> for random
    weights and vectors; hence the normal form M^dag M is Hermitian with <v, M^dag M v> = |M v|^2."""
    lat, X, N = _fields(dims)
    o = make(dims, X, N)
    rng = np.random.default_rng(19)
    W = _rand_vec(rng, o.pc_num_weights) * 0.3
    u, v = hi.gaussian_rhs(lat, 40), hi.gaussian_rhs(lat, 41)
    lhs, rhs = np.vdot(u, o.pc_forward(W, v)), np.vdot(o.pc_adjoint(W, u), v)
    e1 = abs(lhs - rhs) / abs(lhs)
    Mv = o.pc_forward(W, v)
    q = np.vdot(v, o.pc_normal(W, v))
    e2 = abs(q - np.vdot(Mv, Mv).real) / np.vdot(Mv, Mv).real
    return max(e1, e2) <= tol, f"adjoint {e1:.1e}, normal {e2:.1e}"


def pin_network_normal_gradient_fd(make, dims=(4, 4, 4, 4), n_checks=16, tol=1e-6):
    """The normal-form loss gradient equals central finite differences in Re W and Im W, and with
    identity weights (M^dag M = 1) the normal-form loss equals the plain one."""
    lat, X, N = _fields(dims)
    o = make(dims, X, N)
    rng = np.random.default_rng(23)
    W = _rand_vec(rng, o.pc_num_weights) * 0.3
    r = np.stack([hi.gaussian_rhs(lat, 50 + k) for k in range(2)])
    e = np.stack([hi.gaussian_rhs(lat, 60 + k) for k in range(2)])
    mass = 0.3
    _, g = o.pc_loss_grad_normal(W, r, e, mass)
    h = 1e-5
    worst = 0.0
    for i in rng.choice(W.size, n_checks, replace=False):
        for unit, comp in ((1.0, g[i].real), (1j, g[i].imag)):
            Wp, Wm = W.copy(), W.copy()
            Wp[i] += unit * h
            Wm[i] -= unit * h
            fd = (o.pc_loss_grad_normal(Wp, r, e, mass, False)[0]
                  - o.pc_loss_grad_normal(Wm, r, e, mass, False)[0]) / (2 * h)
            worst = max(worst, abs(fd - comp) / max(abs(comp), 1e-3 * np.abs(g).max()))
    Wi = network_weights_identity()
    li, lp = o.pc_loss_grad_normal(Wi, r, e, mass, False)[0], o.pc_loss_grad(Wi, r, e, mass, False)[0]
    ident = abs(li - lp) / lp
    return worst <= tol and ident <= 1e-13, f"worst rel {worst:.2e}, identity {ident:.1e}"



def _fcg_iterates(o, W, b, mass, kmax, form):
    """x_1 .. x_kmax of the oracle's flexible CG (one run per k: the runs are deterministic, so
    the k-iteration run ends at the k-th iterate of any longer one)."""
    return [o.fcg(W, b, mass, tol=1e-300, max_iter=k, form=form)[0].ravel() for k in range(1, kmax + 1)]


def pin_fcg_normal_form_is_pcg(make, dims=(4, 4, 4, 6), mass=0.1, kmax=8, tol=1e-9):
    """With a fixed Hermitian positive-definite preconditioner P flexible CG is preconditioned CG
    (Notay 2000): with P = M^dag M of random weights (assembled densely column by column from the
    oracle's network, which its own pins tie down) the oracle's iterates x_1..x_8 equal those of
    textbook PCG on the dense matrices, z = P r, alpha = <r, z>/<p, A p>, beta = <r', z'>/<r, z>."""
    lat, X, N = _fields(dims)
    o = make(dims, X, N)
    rng = np.random.default_rng(29)
    W = _rand_vec(rng, o.pc_num_weights) * 0.3
    m = 3 * lat.half_volume
    P = np.empty((m, m), dtype=np.complex128)
    for j in range(m):
        e = np.zeros(m, dtype=np.complex128)
        e[j] = 1.0
        P[:, j] = o.pc_normal(W, e.reshape(-1, 3)).ravel()
    A = dense.a_matrix(dims, X, N, mass).toarray()
    b = hi.gaussian_rhs(lat, 6).ravel()
    x = np.zeros(m, dtype=np.complex128)
    r = b.copy()
    z = P @ r
    p = z.copy()
    rz = np.vdot(r, z)
    want = []
    for _ in range(kmax):
        Ap = A @ p
        alpha = rz / np.vdot(p, Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        z = P @ r
        rz_new = np.vdot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
        want.append(x.copy())
    got = _fcg_iterates(o, W, b.reshape(-1, 3), mass, kmax, form=1)
    worst = max(_rel(g, w) for g, w in zip(got, want))
    return worst <= tol, f"max rel diff of x_1..x_{kmax} {worst:.1e}"


def pin_fcg_conjugacy(make, dims=(4, 4, 4, 6), mass=0.1, kmax=8, tol=1e-9):
    """The two defining properties of flexible CG truncated to one direction (Notay 2000), which
    hold for any preconditioner, here the raw network M of random weights (neither Hermitian nor
    constant in its effect): alpha makes the new residual orthogonal to the step,
    <x_k - x_{k-1}, b - A x_k> = 0, and beta makes consecutive steps A-orthogonal,
    <x_k - x_{k-1}, A (x_{k+1} - x_k)> = 0.  Checked from the iterates alone with the dense A."""
    lat, X, N = _fields(dims)
    o = make(dims, X, N)
    rng = np.random.default_rng(31)
    W = _rand_vec(rng, o.pc_num_weights) * 0.3
    A = dense.a_matrix(dims, X, N, mass).toarray()
    b = hi.gaussian_rhs(lat, 7).ravel()
    xs = [np.zeros_like(b)] + _fcg_iterates(o, W, b.reshape(-1, 3), mass, kmax + 1, form=0)
    d = [xs[k] - xs[k - 1] for k in range(1, kmax + 2)]          # d[k-1] is the step of iteration k
    worst_r, worst_a = 0.0, 0.0
    for k in range(1, kmax + 1):
        rk = b - A @ xs[k]
        worst_r = max(worst_r, abs(np.vdot(d[k - 1], rk)) / (np.linalg.norm(d[k - 1]) * np.linalg.norm(rk)))
        Ad = A @ d[k]
        worst_a = max(worst_a, abs(np.vdot(d[k - 1], Ad)) / (np.linalg.norm(d[k - 1]) * np.linalg.norm(Ad)))
    return max(worst_r, worst_a) <= tol, f"residual-step {worst_r:.1e}, A-conjugacy {worst_a:.1e}"

ALL_PINS = [
    pin_matrix_form, pin_anti_hermitian, pin_gauge_covariance, pin_free_field_plane_waves,
    pin_free_field_spectrum, pin_cg_dense_solve, pin_cg_free_field_exact,
    pin_multishift_dense_solve, pin_multishift_free_field_exact, pin_trace_z2_unbiased, pin_condensate_identity,
    pin_network_special_weights, pin_network_covariance, pin_network_gradient_fd, pin_network_loss_zero_at_inverse,
    pin_fcg_identity_is_cg, pin_network_adjoint, pin_network_normal_gradient_fd, pin_fcg_normal_form_is_pcg,
    pin_fcg_conjugacy,
]
