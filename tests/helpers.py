"""Independent textbook helpers for pinning the oracle (numpy only).

These re-derive facts from first principles -- dense H by block expansion,
GF(2) elimination, brute-force maximum likelihood -- and never call the
oracle's encoder or decoder.
"""
import numpy as np


def dense_h(hbm: np.ndarray, z: int) -> np.ndarray:
    """Binary H of eq. (2): block (i, j) with s >= 0 is the Z x Z identity with
    its columns cyclically shifted by s, H[iZ + r][jZ + (r + s) % Z] = 1."""
    mb, nb = hbm.shape
    H = np.zeros((mb * z, nb * z), dtype=np.uint8)
    for i in range(mb):
        for j in range(nb):
            s = int(hbm[i, j])
            if s < 0:
                continue
            for r in range(z):
                H[i * z + r, j * z + (r + s) % z] = 1
    return H


def gf2_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve A x = b over GF(2) for square invertible A (Gauss-Jordan)."""
    A = (A.copy() & 1).astype(np.uint8)
    b = (b.copy() & 1).astype(np.uint8)
    n = A.shape[0]
    for col in range(n):
        piv = None
        for r in range(col, n):
            if A[r, col]:
                piv = r
                break
        if piv is None:
            raise ValueError("singular over GF(2)")
        if piv != col:
            A[[col, piv]] = A[[piv, col]]
            b[[col, piv]] = b[[piv, col]]
        rows = np.nonzero(A[:, col])[0]
        for r in rows:
            if r != col:
                A[r] ^= A[col]
                b[r] ^= b[col]
    return b


def gf2_encode(hbm: np.ndarray, z: int, info: np.ndarray) -> np.ndarray:
    """Systematic codeword [s | p] with H_p p = H_s s (textbook elimination)."""
    H = dense_h(hbm, z)
    mb, nb = hbm.shape
    k = (nb - mb) * z
    Hs, Hp = H[:, :k], H[:, k:]
    rhs = (Hs.astype(np.int64) @ info.astype(np.int64)) & 1
    p = gf2_solve(Hp, rhs.astype(np.uint8))
    return np.concatenate([info.astype(np.uint8), p])


def all_codewords(hbm: np.ndarray, z: int) -> np.ndarray:
    """Every codeword of a tiny code, by brute force over all 2^N words."""
    H = dense_h(hbm, z)
    n = H.shape[1]
    words = ((np.arange(1 << n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    syn = (words.astype(np.int64) @ H.T.astype(np.int64)) & 1
    return words[~syn.any(axis=1)]


def unpack_bits(hard: np.ndarray, n: int) -> np.ndarray:
    hard = np.ascontiguousarray(hard, dtype=np.uint32)
    by = hard.view(np.uint8).reshape(hard.shape[0], -1)
    return np.unpackbits(by, axis=1, bitorder="little")[:, :n]
