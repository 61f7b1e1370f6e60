"""The test-side helpers that certify a plan's low-rank fit at sizes the oracle's SVD cannot
reach (CPU): the streamed Lambda^T Lambda products equal the dense ones, and the top-R
subspace certificate accepts the oracle's own SVD subspace and rejects subspaces that miss
a top singular direction or are not invariant."""
import numpy as np

import oracle as O
from tests import _ref as R


def _small():
    w = R.workload("uca8", 4, 29)  # 2069 cells, L = 300
    dt, Np, lags, perm = R.geometry("uca8", 4, 29)
    Lam = O.interp_matrix(dt, w["fs"], lags)[:, perm]
    return w, dt, lags, perm, Lam


def test_gram_apply_equals_the_dense_product():
    w, dt, lags, perm, Lam = _small()
    Y = np.random.default_rng(1).standard_normal((Lam.shape[1], 5))
    got = R.gram_apply(dt, w["fs"], lags, perm, Y, rows=97, workers=3)
    want = Lam.T @ (Lam @ Y)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_certificate_accepts_the_top_subspace_and_rejects_others():
    w, dt, lags, perm, Lam = _small()
    U, s, Vt = np.linalg.svd(Lam, full_matrices=False)
    R_ = 16
    assert s[R_ - 1] > s[R_] * (1 + 1e-3)  # a gap at this rank

    def apply(Y):
        return Lam.T @ (Lam @ Y)

    V = Vt[:R_].T
    ritz, resid, mu = R.top_subspace_certificate(apply, V.astype(np.float32))
    assert resid <= 1e-6
    assert np.allclose(np.sqrt(ritz), s[:R_], rtol=1e-6)
    assert mu < ritz[-1] * (1 - 1e-6)
    assert mu <= s[R_] ** 2 * (1 + 1e-9) and mu >= 0.5 * s[R_] ** 2
    # an invariant subspace that is not the top one: singular directions 2..R+1
    ritz, resid, mu = R.top_subspace_certificate(apply, Vt[1:R_ + 1].T)
    assert resid <= 1e-10 and mu >= ritz[-1]
    # a subspace that is not invariant: the top one rotated slightly towards direction 40
    Vb = Vt[:R_].T.copy()
    Vb[:, 3] = np.cos(1e-2) * Vb[:, 3] + np.sin(1e-2) * Vt[40]
    ritz, resid, mu = R.top_subspace_certificate(apply, Vb)
    assert resid > 1e-5
