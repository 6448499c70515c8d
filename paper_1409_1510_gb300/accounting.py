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
