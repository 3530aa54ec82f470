"""Round schedule of the thread-block projection with eigenvectors in
registers (csrc/jacobi_reg.cuh), checked on the CPU in float64.

That kernel runs the same two-sided Jacobi (Brent-Luk round-robin ordering,
rotations in Rutishauser's form) as the shared-memory kernel, but reorganises
each round:
  * the rotation of pair k for round r + 1 is formed by the one pair-block of
    round r that produces the entry (sigma^-1(2k+1), sigma^-1(2k)), from that
    block's output and the two diagonals it touches (diagonal -/+ t a_pq);
  * row i of V is split over four parts of contiguous storage pairs; after a
    round the even columns move one pair up and the odd ones one pair down
    (position 0 fixed, 1 -> 2, S-2 -> S-1), each part passing one value to each
    neighbour.
This test replays both organisations with the same formulas and asserts that
they agree bit for bit after every round, that every pair has exactly one
producer block, and that the sweeps converge to the eigendecomposition.  Host
only: no GPU call."""
import numpy as np
import pytest


def _sigma(S):
    K, R = S // 2, S - 1

    def circ_index(p):
        return p // 2 - 1 if p % 2 == 0 else K - 1 + (K - 1 - (p - 1) // 2)

    def circ_pos(c):
        return 2 * (c + 1) if c < K - 1 else 2 * (K - 1 - (c - (K - 1))) + 1

    return [0] + [circ_pos((circ_index(p) + 1) % R) for p in range(1, S)]


def _schur(app, aqq, apq, tol):
    """(tau, sin, t a_pq) of the 2x2 symmetric Schur step; zeros below tol."""
    if abs(apq) <= tol:
        return 0.0, 0.0, 0.0
    zeta = 0.5 * (aqq - app)
    t = np.copysign(1.0, zeta) * apq / (abs(zeta) + np.hypot(zeta, apq))
    c = 1.0 / np.sqrt(1.0 + t * t)
    s = t * c
    return s / (1.0 + c), s, t * apq


def _rot_rows(b0, b1, tau, s):
    return b0 - s * (b1 + tau * b0), b1 + s * (b0 - tau * b1)


class _Layout:
    def __init__(self, S):
        self.S, self.K = S, S // 2
        self.sig = _sigma(S)

    def phys(self, i):
        return self.K + (i >> 1) if i & 1 else i >> 1

    def pos(self, r, c):  # lower-triangle storage key (physical row, column)
        r, c = max(r, c), min(r, c)
        return self.phys(r), self.phys(c)


def _blocks(L):
    """Lower pair-blocks (I, J) and, for the producers, (pair, entry)."""
    K = L.K
    out = []
    for I in range(K):
        for J in range(I + 1):
            prod = None
            if I != J:
                if (I, J) == (1, 0):
                    prod = (0, (1, 0))
                elif (I, J) == (2, 0):
                    prod = (1, (1, 1))
                elif (I, J) == (K - 1, K - 2):
                    prod = (K - 1, (0, 0))
                elif J >= 1 and I == J + 2 and J + 1 <= K - 2:
                    prod = (J + 1, (1, 0))
            out.append((I, J, prod))
    return out


def _round_reference(L, A, V, tol):
    """One round of the shared-memory organisation: rotations from the current
    diagonal blocks, every rotated entry stored at its sigma-permuted place."""
    K, sig = L.K, L.sig
    rot = [_schur(A[L.pos(2 * k, 2 * k)], A[L.pos(2 * k + 1, 2 * k + 1)], A[L.pos(2 * k + 1, 2 * k)], tol)
           for k in range(K)]
    An, Vn = {}, np.empty_like(V)
    for I, J, _ in _blocks(L):
        r0, r1, c0, c1 = 2 * I, 2 * I + 1, 2 * J, 2 * J + 1
        if I == J:
            t = rot[I][2]
            rotated = t != 0.0 or rot[I][1] != 0.0
            An[L.pos(sig[r0], sig[r0])] = A[L.pos(r0, r0)] - t
            An[L.pos(sig[r1], sig[r0])] = 0.0 if rotated else A[L.pos(r1, r0)]
            An[L.pos(sig[r1], sig[r1])] = A[L.pos(r1, r1)] + t
            continue
        (ui, si, _), (uj, sj, _) = rot[I], rot[J]
        q00, q10 = _rot_rows(A[L.pos(r0, c0)], A[L.pos(r1, c0)], ui, si)
        q01, q11 = _rot_rows(A[L.pos(r0, c1)], A[L.pos(r1, c1)], ui, si)
        o00, o01 = _rot_rows(q00, q01, uj, sj)
        o10, o11 = _rot_rows(q10, q11, uj, sj)
        for (r, c), v in (((r0, c0), o00), ((r0, c1), o01), ((r1, c0), o10), ((r1, c1), o11)):
            An[L.pos(sig[r], sig[c])] = v
    for k in range(K):
        u, s, _ = rot[k]
        a, b = _rot_rows(V[:, 2 * k], V[:, 2 * k + 1], u, s)
        Vn[:, sig[2 * k]], Vn[:, sig[2 * k + 1]] = a, b
    return An, Vn


def _parts(K):
    base, rem = K // 4, K % 4
    return [(g * base + min(g, rem), base + (1 if g < rem else 0)) for g in range(4)]


def _round_register(L, A, parts, rot, tol):
    """One round of the register organisation: rotations from the table, the
    producer blocks forming the next table, V rows shifted between parts."""
    K, sig = L.K, L.sig
    An, nxt = {}, [None] * K
    for I, J, prod in _blocks(L):
        r0, r1, c0, c1 = 2 * I, 2 * I + 1, 2 * J, 2 * J + 1
        if I == J:
            t = rot[I][2]
            rotated = t != 0.0 or rot[I][1] != 0.0
            An[L.pos(sig[r0], sig[r0])] = A[L.pos(r0, r0)] - t
            An[L.pos(sig[r1], sig[r0])] = 0.0 if rotated else A[L.pos(r1, r0)]
            An[L.pos(sig[r1], sig[r1])] = A[L.pos(r1, r1)] + t
            continue
        (ui, si, ti), (uj, sj, tj) = rot[I], rot[J]
        q00, q10 = _rot_rows(A[L.pos(r0, c0)], A[L.pos(r1, c0)], ui, si)
        q01, q11 = _rot_rows(A[L.pos(r0, c1)], A[L.pos(r1, c1)], ui, si)
        o00, o01 = _rot_rows(q00, q01, uj, sj)
        o10, o11 = _rot_rows(q10, q11, uj, sj)
        out = {(0, 0): o00, (0, 1): o01, (1, 0): o10, (1, 1): o11}
        for (dr, dc), v in out.items():
            An[L.pos(sig[2 * I + dr], sig[2 * J + dc])] = v
        if prod is not None:
            k, (ro, co) = prod
            a, b = 2 * J + co, 2 * I + ro  # the entry (b, a) becomes (2k+1, 2k)
            assert sig[a] == 2 * k and sig[b] == 2 * k + 1
            app = A[L.pos(a, a)] + (tj if co else -tj)
            aqq = A[L.pos(b, b)] + (ti if ro else -ti)
            nxt[k] = _schur(app, aqq, out[(ro, co)], tol)
    for row in parts:
        for g, (k0, n, ve, vo) in enumerate(row):
            for j in range(n):
                u, s, _ = rot[k0 + j]
                ve[j], vo[j] = _rot_rows(ve[j], vo[j], u, s)
        sends = [(ve[n - 1], vo[0]) for (k0, n, ve, vo) in row]
        for g, (k0, n, ve, vo) in enumerate(row):
            e0, o0 = ve[0], vo[0]
            ve[1:n] = ve[0:n - 1].copy()
            ve[0] = sends[g - 1][0] if g > 0 else e0
            if g == 0:
                ve[1] = o0
            vo[0:n - 1] = vo[1:n].copy()
            vo[n - 1] = sends[g + 1][1] if g < 3 else sends[g][0]
    return An, nxt


def _setup(S, seed):
    rng = np.random.default_rng(seed)
    W = rng.standard_normal((S, S))
    W = W + W.T
    L = _Layout(S)
    A = {L.pos(a, b): W[a, b] for a in range(S) for b in range(a + 1)}
    tol = 1e-14 * np.linalg.norm(W)
    return W, L, A, tol


def _register_state(S, L, A, tol):
    """V = I split over the four parts of every row, and the first round's
    rotations (formed from the diagonal blocks before the first round)."""
    parts = [[(k0, n, np.array([1.0 if i == 2 * (k0 + j) else 0.0 for j in range(n)]),
               np.array([1.0 if i == 2 * (k0 + j) + 1 else 0.0 for j in range(n)])) for k0, n in _parts(S // 2)]
             for i in range(S)]
    rot = [_schur(A[L.pos(2 * k, 2 * k)], A[L.pos(2 * k + 1, 2 * k + 1)], A[L.pos(2 * k + 1, 2 * k)], tol)
           for k in range(S // 2)]
    return parts, rot


def _v_from_parts(S, parts):
    V = np.zeros((S, S))
    for i, row in enumerate(parts):
        for k0, n, ve, vo in row:
            for j in range(n):
                V[i, 2 * (k0 + j)], V[i, 2 * (k0 + j) + 1] = ve[j], vo[j]
    return V


@pytest.mark.parametrize("S", [36, 40, 44, 48, 52, 56, 60, 64])
def test_every_pair_has_one_producer(S):
    L = _Layout(S)
    pairs = sorted(p[0] for _, _, p in _blocks(L) if p is not None)
    assert pairs == list(range(S // 2))


@pytest.mark.parametrize("S", [36, 44, 52, 64])
def test_register_rounds_equal_reference_rounds(S):
    W, L, A, tol = _setup(S, S)
    Ar, Vr = dict(A), np.eye(S)
    parts, rot = _register_state(S, L, A, tol)
    An = dict(A)
    for _ in range(S - 1):  # one sweep
        Ar, Vr = _round_reference(L, Ar, Vr, tol)
        An, rot = _round_register(L, An, parts, rot, tol)
        assert Ar == An
        np.testing.assert_array_equal(_v_from_parts(S, parts), Vr)


def test_register_sweeps_converge_to_the_eigendecomposition():
    S = 40
    W, L, A, tol = _setup(S, 7)
    parts, rot = _register_state(S, L, A, tol)
    for _ in range(9 * (S - 1)):  # nine sweeps; each returns the storage order to the identity
        A, rot = _round_register(L, A, parts, rot, tol)
    lam = np.array([A[L.pos(i, i)] for i in range(S)])
    off = max(abs(A[L.pos(a, b)]) for a in range(S) for b in range(a))
    V = _v_from_parts(S, parts)
    assert off <= 1e-12 * np.linalg.norm(W)
    np.testing.assert_allclose(np.sort(lam), np.linalg.eigvalsh(W), atol=1e-11 * np.linalg.norm(W))
    np.testing.assert_allclose(V @ np.diag(lam) @ V.T, W, atol=1e-11 * np.linalg.norm(W))
    np.testing.assert_allclose(V.T @ V, np.eye(S), atol=1e-12)
