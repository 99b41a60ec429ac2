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
