"""Shared test helpers: packed-triangle indexing and the normalised error
metric max |dV_ij| / sqrt(V_ii V_jj) used for every floating-point tolerance."""
import numpy as np


def tri_index(N):
    i, j = np.tril_indices(N)
    order = np.argsort(i * (i + 1) // 2 + j)
    return i[order], j[order]


def diag_bl(N):
    n = np.arange(N)
    return n * (n + 1) // 2 + n


def norm_err(V, Vref, N):
    """V, Vref: [..., NB] complex.  Normalised by the reference autocorrelations."""
    V = np.asarray(V).reshape(-1, N * (N + 1) // 2)
    Vref = np.asarray(Vref).reshape(-1, N * (N + 1) // 2)
    ii, jj = tri_index(N)
    auto = Vref[:, diag_bl(N)].real
    den = np.sqrt(np.maximum(auto[:, ii] * auto[:, jj], 1e-300))
    return float(np.max(np.abs(V - Vref) / den))


def norm_err_subset(V_full_at, Vref_sub, idx):
    """Sampled parity: V_full_at(i, j) -> value from the full-size result for
    global inputs (i, j); Vref_sub: oracle V over the input subset idx."""
    n = len(idx)
    ii, jj = tri_index(n)
    Vref = np.asarray(Vref_sub).reshape(-1, n * (n + 1) // 2)
    got = np.stack([V_full_at(c, idx[a], idx[b]) for c in range(Vref.shape[0]) for a, b in zip(ii, jj)])
    got = got.reshape(Vref.shape)
    auto = Vref[:, diag_bl(n)].real
    den = np.sqrt(auto[:, ii] * auto[:, jj])
    return float(np.max(np.abs(got - Vref) / den))
