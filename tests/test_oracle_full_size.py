"""The oracle's TLR integrand (Algorithm 6) pinned at the bench's full size, n = 65,536
with 512-variable tiles, on a factor whose integrand has a closed form per sample
(tests.helpers.sources_targets_factor): infinite limits on alternate tiles make their
variables plain normal quantiles of the lattice values, identity diagonal tiles elsewhere
leave one log Phi per variable, so every per-sample value is a direct sum that does not go
through the tile recursion.  A wrong tile offset, a transposed U or V, a sign of the shift
or a shift applied to the wrong tiles changes the values."""
from __future__ import annotations

import math

import numpy as np
from scipy import stats

from oracle import sov
from tests.helpers import closed_form_logf, sources_targets_factor


def test_tlr_integrand_full_size_closed_form():
    n, m, S = 65_536, 512, 6
    F, b = sources_targets_factor(n, m, seed=11)
    W = np.random.default_rng(12).uniform(1e-6, 1.0 - 1e-6, (n, S))
    a = np.full((n, 1), -np.inf)
    got = sov.tlrmvn(F, a, b[:, None], W)
    want = closed_form_logf(F, b, W)
    assert np.all(np.isfinite(want)) and np.all(want < -100.0)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=0.0)


def test_closed_form_sees_the_low_rank_push():
    """The same problem with the low-rank factors dropped gives other values, so the pin
    above depends on the shifts (it is not satisfied by the diagonal tiles alone)."""
    n, m, S = 4_096, 512, 4
    F, b = sources_targets_factor(n, m, seed=13)
    W = np.random.default_rng(14).uniform(1e-6, 1.0 - 1e-6, (n, S))
    a = np.full((n, 1), -np.inf)
    full = sov.tlrmvn(F, a, b[:, None], W)
    for k in F.U:
        F.U[k] = F.U[k][:, :0]
        F.V[k] = F.V[k][:, :0]
    bare = sov.tlrmvn(F, a, b[:, None], W)
    assert np.min(np.abs(full - bare)) > 1.0


def test_tlr_student_t_full_size_closed_form():
    """Algorithm 7 at the same size: the target limits scale by chi_nu^-1(w0)/sqrt(nu), w0 the
    lattice value of coordinate n (SciPy's chi quantile here, not the oracle's)."""
    n, m, S, nu = 65_536, 512, 4, 7.0
    F, b = sources_targets_factor(n, m, seed=15)
    Wall = np.random.default_rng(16).uniform(1e-6, 1.0 - 1e-6, (S, n + 1))
    got = sov.per_sample_logp(F, None, F.perm, np.full(n, -np.inf), b, nu, Wall)
    rs = stats.chi.ppf(Wall[:, n], nu) / math.sqrt(nu)
    want = closed_form_logf(F, b, Wall[:, :n].T, rs)
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=0.0)
