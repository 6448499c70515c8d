"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check that the pins catch
every one of them: a dropped term, a wrong sign, a wrong hop length or site, a transposed
operand, a wrong mass term and a wrong CG coefficient, a missing conjugation in the adjoint
network, a dropped term of the normal-form gradient, wrong multi-shift recurrences, a wrong trace estimator or biased noise,
and a Fletcher-Reeves numerator, a misplaced conjugate or a missing adjoint in flexible CG."""
import os
import tempfile

import pytest

import oracle
import oracle.build as obuild
import oracle_pins as pins

MUTANTS = {
    "drop_backward_naik": (
        "w[a] = c_sub(w[a], c_mul(c_conj(link(N, V, mu, xm3, b, a)), vin(ctx, xm3, b)));", ""),
    "sign_backward_fat": (
        "w[a] = c_sub(w[a], c_mul(c_conj(link(X, V, mu, xm1, b, a)), vin(ctx, xm1, b)));",
        "w[a] = c_add(w[a], c_mul(c_conj(link(X, V, mu, xm1, b, a)), vin(ctx, xm1, b)));"),
    "naik_hop_two": ("long xp3 = hop(L, x, mu, +3)", "long xp3 = hop(L, x, mu, +2)"),
    "conj_not_dagger": (
        "c_mul(c_conj(link(X, V, mu, xm1, b, a)), vin(ctx, xm1, b))",
        "c_mul(c_conj(link(X, V, mu, xm1, a, b)), vin(ctx, xm1, b))"),
    "backward_link_wrong_site": (
        "c_mul(c_conj(link(N, V, mu, xm3, b, a)), vin(ctx, xm3, b))",
        "c_mul(c_conj(link(N, V, mu, xm1, b, a)), vin(ctx, xm3, b))"),
    "forward_link_transposed": (
        "c_mul(link(X, V, mu, x, a, b), vin(ctx, xp1, b))",
        "c_mul(link(X, V, mu, x, b, a), vin(ctx, xp1, b))"),
    "mass_not_squared": ("w[i] = mass * mass * v[i] - w[i];", "w[i] = mass * v[i] - w[i];"),
    "cg_beta_inverted": ("double beta = rr_new / rr;", "double beta = rr / rr_new;"),
    "network_adjoint_sign": ("cplx wc = {w[0], -w[1]};", "cplx wc = {w[0], w[1]};"),
    "network_backward_hop_forward": ("long y = hop(L, x, mu, -step);", "long y = hop(L, x, mu, step);"),
    "network_adjoint_not_conjugated": ("cplx wc = c_conj((cplx){w[0], w[1]});", "cplx wc = (cplx){w[0], w[1]};"),
    "multishift_zeta_shift_sign": ("(1.0 + s * alpha)", "(1.0 - s * alpha)"),
    "multishift_beta_not_squared": ("double beta_j = beta_base * ratio * ratio;", "double beta_j = beta_base * ratio;"),
    "multishift_alpha_ratio_inverted": ("double alpha_j = alpha * zeta_new[j] / zeta[j];",
                                        "double alpha_j = alpha * zeta[j] / zeta_new[j];"),
    "trace_estimator_uses_x_not_eta": ("double v = dot(eta, x, n).re;", "double v = dot(x, x, n).re;"),
    "noise_not_symmetric": ("(z >> 63) ? -1.0 : 1.0", "(z >> 62) ? -1.0 : 1.0"),
    "normal_loss_missing_n_dag_term": ("oracle_pc_backward(L, X, N, W, gy, h, grad);        /* through N^dag */",
                                       "/* dropped */"),
    "fcg_beta_fletcher_reeves": ("for (long i = 0; i < 2 * n; i++) Ap[i] = r[i] - r_old[i];",
                                 "for (long i = 0; i < 2 * n; i++) Ap[i] = r[i];"),
    "fcg_beta_conjugate_misplaced": ("beta = c_scale(1.0 / den, c_mul(num, c_conj(rp_old)));",
                                     "beta = c_scale(1.0 / den, c_mul(c_conj(num), rp_old));"),
    "fcg_alpha_conjugated": ("cplx alpha = c_scale(1.0 / pAp, pr);", "cplx alpha = c_scale(1.0 / pAp, c_conj(pr));"),
    "fcg_normal_form_without_adjoint": ("oracle_pc_adjoint(L, X, N, W, Ap, z);", "memcpy(z, Ap, sizeof(double) * n * 2);"),
}


@pytest.fixture(scope="module")
def source():
    with open(obuild.SOURCE) as f:
        return f.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, source):
    old, new = MUTANTS[name]
    assert source.count(old) == 1, f"mutation site for {name} not found exactly once"
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "mutant.c")
        with open(src, "w") as f:
            f.write(source.replace(old, new))
        so = obuild.build(force=True, output=os.path.join(d, "mutant.so"), source=src)

        def make(dims, X, N):
            return oracle.Oracle(dims, X, N, so_path=so)

        caught = []
        for pin in pins.ALL_PINS:
            try:
                ok, _ = pin(make)
            except Exception:  # a crash or a non-finite result also counts as caught
                ok = False
            if not ok:
                caught.append(pin.__name__)
                break
        assert caught, f"no pin caught mutant {name}"
