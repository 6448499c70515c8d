"""Flop and byte accounting of the HISQ Dslash (Table 1, Eq. (3)-(4)).

Per output site and right-hand side the Dslash of Eq. (3) performs 16 complex 3x3
matrix-vector products (9 complex multiplications at 6 flop and 6 complex additions at 2 flop:
66 flop each) and sums the 16 resulting colour vectors (15 additions of 3 complex numbers:
6 flop each): 16*66 + 15*6 = 1146 flop.

Table 1 counts bytes the way the paper's model does: 16 links per site (8 fat, 8 Naik) plus,
for every right-hand side, the 16 neighbour vectors and the output vector (17 colour vectors),
all in single precision, with nothing re-used from caches.  The "compulsory" model used for the
roofline reads every link and every input vector once and writes the output once.
"""

MATVEC_FLOPS = 9 * 6 + 6 * 2          # one complex 3x3 matrix times colour vector
DSLASH_FLOPS_PER_SITE = 16 * MATVEC_FLOPS + 15 * 3 * 2   # 1146, per output site per RHS
CG_EXTRA_FLOPS_PER_SITE = 72          # m^2 axpy, 2 dots and 3 axpys on one even site per RHS
CG_FLOPS_PER_SITE = 2 * DSLASH_FLOPS_PER_SITE + CG_EXTRA_FLOPS_PER_SITE

LINK_REALS = 18          # full 3x3 complex matrix
VECTOR_REALS = 6         # 3 complex colour components
LINKS_PER_SITE = 16      # 8 fat (4 forward, 4 backward) + 8 Naik


def paper_model_bytes(nrhs: int, naik_reals: int = LINK_REALS, real_bytes: int = 4) -> int:
    """Bytes per output site in the Table 1 model (no re-use of vectors or links)."""
    links = (8 * LINK_REALS + 8 * naik_reals) * real_bytes
    return links + 17 * VECTOR_REALS * real_bytes * nrhs


def paper_model_intensity(nrhs: int, naik_reals: int = LINK_REALS) -> float:
    """Flop/byte of the Dslash in the Table 1 model."""
    return DSLASH_FLOPS_PER_SITE * nrhs / paper_model_bytes(nrhs, naik_reals)


def link_bytes_per_site(link_real_bytes: float, naik_reals: int = LINK_REALS,
                        fat_scale_bytes: float = 0.0) -> float:
    """Stored link bytes read per output site: 8 fat + 8 Naik links (+ a per-site fat scale)."""
    return 8 * LINK_REALS * link_real_bytes + 8 * naik_reals * link_real_bytes + fat_scale_bytes


def compulsory_bytes(nrhs: int, link_real_bytes: float, vector_real_bytes: float,
                     naik_reals: int = LINK_REALS, fat_scale_bytes: float = 0.0,
                     vector_scale_bytes: float = 0.0) -> float:
    """Algorithmic bytes per output site of one even-odd Dslash: every stored link once, each
    input vector once and each output vector once (plus per-(site, RHS) scales if any)."""
    vec = VECTOR_REALS * vector_real_bytes + vector_scale_bytes
    return link_bytes_per_site(link_real_bytes, naik_reals, fat_scale_bytes) + 2 * vec * nrhs


# ---- the whole mixed-precision CG solve (algorithmic bytes per even site and RHS) ----------------
# Storage per colour vector of one site and right-hand side: FP64 48 B, FP32 24 B, FP16 12 B plus
# a 4 B scale, BF16 12 B.  The iterated x and r are FP32 unless the inner precision is FP64.
VECTOR_BYTES = {0: 48.0, 1: 24.0, 2: 16.0, 3: 12.0}
LINK_BYTES_18 = {0: 2 * 8 * 18 * 8.0, 1: 2 * 8 * 18 * 4.0, 2: 2 * 8 * 18 * 2.0 + 8.0, 3: 2 * 8 * 18 * 2.0 + 8.0}


def cg_iteration_bytes(prec: int, nrhs: int = 1) -> float:
    """One iteration of a bundle, per even site, with 18-real links read once for the bundle:
    t = D_oe p (links; p, t), A p = m^2 p - D_eo t (links; t, p, Ap), x += alpha p and
    r -= alpha A p (p, Ap read; x, r read and written), p = r + beta p (r read; p read and
    written): 2 links + nrhs (9 P + 5 Q) bytes."""
    P = VECTOR_BYTES[prec]
    Q = VECTOR_BYTES[0] if prec == 0 else VECTOR_BYTES[1]
    return 2 * LINK_BYTES_18[prec] + nrhs * (9 * P + 5 * Q)


def reliable_update_bytes(prec: int, nrhs: int = 1) -> float:
    """One FP64 residual recomputation of a bundle, per even site: x_hi += x (x read and zeroed,
    x_hi read and written), t = D_oe x_hi (FP64 links; x_hi, t), r = b - m^2 x_hi + D_eo t (FP64
    links; t, x_hi, b read; r written in the iterated precision)."""
    Q = VECTOR_BYTES[0] if prec == 0 else VECTOR_BYTES[1]
    L64 = LINK_BYTES_18[0]
    return 2 * L64 + nrhs * ((2 * Q + 96.0) + 96.0 + (144.0 + Q))


def cg_setup_bytes(prec: int, nrhs: int = 1) -> float:
    """Setup of a bundle per even site: b read; x_hi, x, r, p written."""
    P = VECTOR_BYTES[prec]
    Q = VECTOR_BYTES[0] if prec == 0 else VECTOR_BYTES[1]
    return nrhs * (96.0 + 2 * Q + P)


def cg_solve_bytes(prec: int, half_volume: int, iterations: int, reliable_updates: int, nrhs: int = 1) -> float:
    """Algorithmic bytes of one bundle solve whose nrhs right-hand sides all ran `iterations`
    iterations and `reliable_updates` FP64 recomputations."""
    per = (cg_setup_bytes(prec, nrhs) + iterations * cg_iteration_bytes(prec, nrhs)
           + reliable_updates * reliable_update_bytes(prec, nrhs))
    return per * half_volume


def multishift_iteration_bytes(prec: int, live_shifts: int) -> float:
    """One shared multi-shift iteration per even site (one right-hand side): t = D_oe p (links;
    p, t), A p = m^2 p - D_eo t (links; t, p, Ap), the update pass (r read and written, Ap read;
    per live shift x_j and p_j read and written) and the direction pass (r read, p read and
    written): 2 links + 8 P + 3 Q + 4 Q per live shift."""
    P = VECTOR_BYTES[prec]
    Q = VECTOR_BYTES[0] if prec == 0 else VECTOR_BYTES[1]
    return 2 * LINK_BYTES_18[prec] + 8 * P + 3 * Q + 4 * Q * live_shifts


def recompute_flops(half_volume: int, reliable_updates: int) -> float:
    """Algorithmic flops of the residual recomputations: two Dslash (1146 flop per site and
    right-hand side each) per recomputation of one right-hand side; the m^2 x and b terms are
    counted with the iteration."""
    return 2.0 * DSLASH_FLOPS_PER_SITE * half_volume * reliable_updates


def bundle_solve_bytes(prec: int, half_volume: int, total_iterations: int, bundle_iterations: int,
                       reliable_updates: int, recompute_passes: int, nrhs: int) -> float:
    """Algorithmic bytes of the bundle solves of one hisq_cg_solve: the links once per bundle
    iteration (both Dslash), the vectors of every right-hand side once per iteration it ran
    (9 P + 5 Q), the FP64-accurate links (double-single or FP64: 8 bytes per real) once per
    recomputation pass (both Dslash), the vectors of every recomputed right-hand side, and the
    setup of every right-hand side."""
    P = VECTOR_BYTES[prec]
    Q = VECTOR_BYTES[0] if prec == 0 else VECTOR_BYTES[1]
    L64 = LINK_BYTES_18[0]
    per_rhs_recompute = (2 * Q + 96.0) + 96.0 + (144.0 + Q)
    total = (bundle_iterations * 2 * LINK_BYTES_18[prec] + total_iterations * (9 * P + 5 * Q)
             + recompute_passes * 2 * L64 + reliable_updates * per_rhs_recompute + nrhs * cg_setup_bytes(prec))
    return total * half_volume
