"""Test-only helpers: pack the oracle's complex 3x3 matrices into the library's
9-real layout and measure family-wise relative errors."""
import numpy as np

PACK = [(0, 0, "re"), (1, 1, "re"), (2, 2, "re"), (0, 1, "re"), (0, 1, "im"), (0, 2, "re"), (0, 2, "im"),
        (1, 2, "re"), (1, 2, "im")]


def pack(m: np.ndarray) -> np.ndarray:
    """(..., 3, 3) complex Hermitian -> (9, ...) packed reals."""
    out = []
    for a, b, part in PACK:
        v = m[..., a, b]
        out.append(v.real if part == "re" else v.imag)
    return np.stack(out, axis=0)


def unpack(v: np.ndarray) -> np.ndarray:
    """(9, ...) packed reals -> (..., 3, 3) complex Hermitian."""
    shape = v.shape[1:]
    m = np.zeros(shape + (3, 3), complex)
    m[..., 0, 0], m[..., 1, 1], m[..., 2, 2] = v[0], v[1], v[2]
    for (a, b), k in (((0, 1), 3), ((0, 2), 5), ((1, 2), 7)):
        m[..., a, b] = v[k] + 1j * v[k + 1]
        m[..., b, a] = v[k] - 1j * v[k + 1]
    return m


def fro(v: np.ndarray) -> np.ndarray:
    """Frobenius norm of each Hermitian matrix of a (9, N) packed array."""
    return np.sqrt((np.abs(unpack(v)) ** 2).sum(axis=(-1, -2)))


def family_err(got: np.ndarray, ref: np.ndarray, scale: float = None) -> float:
    """max over items of ||got - ref||_F divided by `scale`, by default the
    max over items of ||ref||_F, for (9, N) packed arrays.  Grid quantities
    that are sums with cancellation (fluxes of isotropic species, n - nbar^*,
    H) are measured against the density scale of their summands instead."""
    num = fro(np.asarray(got) - np.asarray(ref)).max()
    den = fro(ref).max() if scale is None else scale
    return float(num / den) if den > 0 else float(num)


def density_scales(grid):
    """(max_j ||n_j||_F, max_j ||nbar_j||_F, max_j (||n_j||_F + ||nbar_j||_F)) of an oracle grid."""
    n = fro(pack(grid["n"]))
    nb = fro(pack(grid["nbar"]))
    return float(n.max()), float(nb.max()), float((n + nb).max())


def oracle_potential(grid, kappa) -> np.ndarray:
    """kappa (n - nbar^*) and kappa (f_i - fbar_i^*) of an oracle grid, as (36, nz)."""
    a0 = pack(grid["n"] - np.conj(grid["nbar"]))
    ai = [pack(grid["f"][:, i] - np.conj(grid["fbar"][:, i])) for i in range(3)]
    return kappa * np.concatenate([a0] + ai, axis=0)


def oracle_moments(grid) -> np.ndarray:
    """(72, nz): n, f_x, f_y, f_z, nbar, fbar_x, fbar_y, fbar_z packed."""
    parts = [pack(grid["n"])] + [pack(grid["f"][:, i]) for i in range(3)]
    parts += [pack(grid["nbar"])] + [pack(grid["fbar"][:, i]) for i in range(3)]
    return np.concatenate(parts, axis=0)


def moment_families(m: np.ndarray):
    """Split a (72, nz) moments array into its 8 (9, nz) families."""
    return [m[9 * i:9 * (i + 1)] for i in range(8)]
