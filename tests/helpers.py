"""Small helpers shared by the tests (no method arithmetic)."""
import numpy as np


def nrmse(y, ref) -> float:
    y = np.asarray(y).reshape(-1)
    ref = np.asarray(ref).reshape(-1)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(y - ref) / (den if den > 0 else 1.0))


def iq_to_complex(q) -> np.ndarray:
    q = np.asarray(q)
    return q[..., 0].astype(np.float64) + 1j * q[..., 1].astype(np.float64)


def complex_to_iq16(z) -> np.ndarray:
    z = np.asarray(z)
    out = np.empty(z.shape + (2,), dtype=np.int16)
    out[..., 0] = z.real
    out[..., 1] = z.imag
    return out


def impulse_x(n_tx, total, positions, amp=(3, -2)):
    x = np.zeros((n_tx, total, 2), dtype=np.int16)
    for t in range(n_tx):
        for p in positions:
            x[t, p, 0] = amp[0] * (t + 1)
            x[t, p, 1] = amp[1]
    return x


# Relative closeness of two tap powers below which a binary32 power (components rounded to binary32,
# one rounded square, one rounded fused multiply-add: at most about 3.5 * 2^-23 relative error) can
# order them either way.  Generous by a factor of about 2.
TOPN_AMBIGUITY = 2.0 ** -20


def topn_selections(H, top_n: int, eps: float = TOPN_AMBIGUITY):
    """Valid top-n selections of one anchor (ranking only, no method arithmetic).

    H: complex128 [n_rx][n_tx][K] anchor.  Returns (base, alts): base bool [n_rx][n_tx][K] is the FP64
    selection (largest |H|^2, ties to the lower index; every tap when top_n is 0 or >= K), and
    alts = {(r, t): [bool[K], ...]} lists, for each link with a near tie at the n-th place, the base
    selection first and then every other selection that differs from it only among taps whose power
    lies within eps (relative) of the n-th largest power, where a lower-precision ranking could order
    them either way.
    """
    import itertools
    H = np.asarray(H)
    n_rx, n_tx, K = H.shape
    base = np.ones((n_rx, n_tx, K), dtype=bool)
    alts = {}
    if not top_n or top_n >= K:
        return base, alts
    for r in range(n_rx):
        for t in range(n_tx):
            p = np.abs(H[r, t]) ** 2
            order = sorted(range(K), key=lambda k: (-p[k], k))
            pn = p[order[top_n - 1]]
            first = np.zeros(K, dtype=bool)
            first[order[:top_n]] = True
            base[r, t] = first
            group = [k for k in range(K) if abs(p[k] - pn) <= eps * pn]
            sure = [k for k in range(K) if p[k] > pn and k not in group]
            need = top_n - len(sure)
            if len(group) <= need:
                continue
            links = [first]
            for pick in itertools.combinations(group, need):
                m = np.zeros(K, dtype=bool)
                m[sure] = True
                m[list(pick)] = True
                if not np.array_equal(m, first):
                    links.append(m)
            alts[(r, t)] = links
    return base, alts
