"""Matrix form of the HISQ Dslash, assembled entry by entry from Eq. (3).

TEST INFRASTRUCTURE ONLY.  An independent statement of the operator used to check the C
oracle: D is assembled as a sparse matrix over (site, colour) with every 3x3 block of Eq. (3)
*added* into place, because on small lattices several hops reach the same neighbour
(on L_mu = 4, x+3mu is x-mu and x+2mu is x-2mu).  Row/column index is 3*lex + colour.
"""
import numpy as np
import scipy.sparse as sp


def _coords(dims):
    lx, ly, lz, lt = dims
    i = np.arange(lx * ly * lz * lt)
    return np.stack([i % lx, (i // lx) % ly, (i // (lx * ly)) % lz, i // (lx * ly * lz)], axis=1)


def _lex(dims, c):
    lx, ly, lz, _ = dims
    return c[:, 0] + lx * (c[:, 1] + ly * (c[:, 2] + lz * c[:, 3]))


def _shifted(dims, mu, step):
    c = _coords(dims)
    c[:, mu] = (c[:, mu] + step) % dims[mu]
    return _lex(dims, c)


def dslash_matrix(dims, fat, naik):
    """Full-lattice D (3V x 3V, CSR): Eq. (3) with links fat, naik [4][V][3][3]."""
    V = int(np.prod(dims))
    X = np.asarray(fat).reshape(4, V, 3, 3)
    N = np.asarray(naik).reshape(4, V, 3, 3)
    rows, cols, vals = [], [], []
    x = np.arange(V)
    a_idx, b_idx = np.meshgrid(np.arange(3), np.arange(3), indexing="ij")

    def add_block(target_sites, blocks, sign):
        # blocks[x][a][b] multiplies v_{target(x), b} into w_{x, a}
        rows.append((3 * x[:, None, None] + a_idx[None]).ravel())
        cols.append((3 * target_sites[:, None, None] + b_idx[None]).ravel())
        vals.append((sign * blocks).ravel())

    for mu in range(4):
        xp1, xm1 = _shifted(dims, mu, 1), _shifted(dims, mu, -1)
        xp3, xm3 = _shifted(dims, mu, 3), _shifted(dims, mu, -3)
        add_block(xp1, X[mu], +1.0)
        add_block(xm1, X[mu][xm1].conj().swapaxes(-1, -2), -1.0)
        add_block(xp3, N[mu], +1.0)
        add_block(xm3, N[mu][xm3].conj().swapaxes(-1, -2), -1.0)
    coo = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                        shape=(3 * V, 3 * V))
    return coo.tocsr()  # duplicate (row, col) entries are summed


def parity_rows(dims, parity):
    """Row indices (3*lex + colour) of the sites of one parity, in even-odd order."""
    c = _coords(dims)
    lex = np.nonzero(c.sum(axis=1) % 2 == parity)[0]
    return (3 * lex[:, None] + np.arange(3)[None]).ravel()


def even_odd_blocks(dims, fat, naik):
    """(D_eo, D_oe) as sparse blocks of the full matrix."""
    D = dslash_matrix(dims, fat, naik)
    e, o = parity_rows(dims, 0), parity_rows(dims, 1)
    return D[e][:, o], D[o][:, e]


def a_matrix(dims, fat, naik, mass):
    """A = m^2 1 - D_eo D_oe on even sites (sparse)."""
    deo, doe = even_odd_blocks(dims, fat, naik)
    n = deo.shape[0]
    return (mass * mass) * sp.identity(n, dtype=np.complex128, format="csr") - deo @ doe
