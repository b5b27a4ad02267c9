"""Canonical form of a stabilizer group, for comparing final tableaus.

Two generating sets of one stabilizer group (the engine's forward
generators from its inverse tableau, the oracle's stabilizer rows) differ
row by row; the reduced row echelon form over the columns x_0..x_{n-1},
z_0..z_{n-1}, with generators multiplied as Paulis (phases tracked mod 4),
is unique for the group.  The group's elements commute, so the order of a
product does not change its phase."""
import numpy as np


def canonical(x, z, r):
    """Generators (-1)^r i^{x.z} X^x Z^z (rows) -> the reduced row echelon
    form of the group they generate, with signs: (x, z, r) arrays."""
    M = np.concatenate([x, z], axis=1).astype(np.uint8)
    n = x.shape[1]
    e = (2 * r.astype(np.int64) + np.sum(x.astype(np.int64) & z, axis=1)) % 4  # P = i^e X^x Z^z
    k = 0
    for col in range(2 * n):
        if k == M.shape[0]:
            break
        cand = np.nonzero(M[k:, col])[0]
        if len(cand) == 0:
            continue
        p = k + int(cand[0])
        M[[k, p]] = M[[p, k]]
        e[[k, p]] = e[[p, k]]
        hit = np.nonzero(M[:, col])[0]
        hit = hit[hit != k]
        if len(hit):
            # row_q <- row_k * row_q: e_q += e_k + 2 popc(z_k & x_q)
            zk = M[k, n:].astype(np.int64)
            e[hit] = (e[hit] + e[k] + 2 * (M[hit, :n].astype(np.int64) @ zk)) % 4
            M[hit] ^= M[k]
        k += 1
    assert k == M.shape[0], "generators are not independent"
    xx, zz = M[:, :n], M[:, n:]
    ph = (e - np.sum(xx.astype(np.int64) & zz, axis=1)) % 4
    assert np.all(ph % 2 == 0), "a generator is not Hermitian"
    return xx, zz, (ph // 2).astype(np.uint8)


