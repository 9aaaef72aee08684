"""Block-reordered TLR Cholesky factor (oracle; test infrastructure only).

Section 3.3 of the paper:

* Algorithm 4 (block reordering, "r"): estimate p_l ~ Phi_m(a_l, b_l; Sigma_ll)
  for every diagonal block, then order the blocks by ascending p_l; a plain
  (TLR) Cholesky factorisation follows.
* Algorithm 5 (iterative block reordering, "rr"): at step j, estimate p_l on
  the current Schur complement Sigma_ll with the current (conditioned) limits
  for every remaining block, bring the block with the smallest estimate to
  position j, take its truncated expectations y_j, factor it, form
  L_ij = Sigma_ij Sigma_jj^-T for the blocks below, shift their limits by
  L_ij y_j, and subtract L_i1j L_j1j^T from the remaining Schur complement.
* p_l and y_j come from univariate conditioning (Trinh & Genz, 2015), an
  O(m^3) pivoted Cholesky that at every step takes the remaining variable with
  the smallest conditional interval probability.  The paper's reordering acts
  both across and inside the diagonal blocks (abstract): the within-block
  order is the pivot order of that univariate conditioning.
* Off-diagonal tiles are stored as U V^T, truncated by adaptive cross
  approximation (ACA) at an absolute tolerance (Section 3.3).  Here ACA uses
  full pivoting on the dense tile and stops when the largest residual entry
  is at most tol (or at the rank cap), and each rank-one term is balanced
  (|u| = |v|).
* Two arithmetics: tlr_factor keeps the Schur complement exact and truncates
  each finished factor tile once; tlr_factor_truncated is the printed form of
  Section 3.3, with the covariance compressed first and every product and
  subtraction truncated.

Readings where the paper is silent (restated in the design notes):
* tlr_factor: the Schur complement is kept dense and exact; only the finished
  factor tiles L_ij are truncated (the paper truncates the Schur tiles too,
  which differs by O(tol); tlr_factor_truncated does that);
* Algorithm 5 overwrites the limits; those conditioned limits steer the
  ordering only, and the integration uses the original limits, permuted;
* ties in argmin/argmax go to the first candidate (lowest position / first
  entry in row-major order).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np
from scipy.linalg import solve_triangular

from . import special

REORDER_NONE = 0
REORDER_BODR = 1
REORDER_RBODR = 2


@dataclass
class UCResult:
    order: np.ndarray   # order[k] = local index placed at position k
    L: np.ndarray       # pivoted Cholesky factor, in the new order (lower)
    y: np.ndarray       # truncated expectations, in the new order
    log_p: float        # log of the univariate-conditioning estimate of Phi_m


def univariate_conditioning(S: np.ndarray, a: np.ndarray, b: np.ndarray) -> UCResult:
    """Univariate conditioning estimate of Phi_m(a, b; S) with its pivot order.

    At step k the remaining variables have conditional standard deviation
    sigma_i and conditional shift s_i given the truncated expectations of the
    variables already placed; the variable with the smallest
    Phi((b_i - s_i)/sigma_i) - Phi((a_i - s_i)/sigma_i) goes next, its
    Cholesky column is formed, and its truncated expectation y_k enters the
    shifts of the rest.  The estimate is the product of the chosen probabilities.
    """
    A = np.array(S, dtype=np.float64, copy=True)
    a = np.array(a, dtype=np.float64, copy=True)
    b = np.array(b, dtype=np.float64, copy=True)
    m = A.shape[0]
    order = np.arange(m)
    s = np.zeros(m)
    L = np.zeros((m, m))
    y = np.zeros(m)
    log_p = 0.0
    for k in range(m):
        var = np.diag(A)[k:].copy()
        if np.any(var <= 0.0):
            raise np.linalg.LinAlgError("covariance block is not positive definite")
        sig = np.sqrt(var)
        at = (a[k:] - s[k:]) / sig
        bt = (b[k:] - s[k:]) / sig
        q = special.log_interval(at, bt)
        i = k + int(np.argmin(q))
        if i != k:
            for arr in (a, b, s, order):
                arr[[k, i]] = arr[[i, k]]
            A[[k, i], :] = A[[i, k], :]
            A[:, [k, i]] = A[:, [i, k]]
            L[[k, i], :k] = L[[i, k], :k]
        lkk = np.sqrt(A[k, k])
        L[k, k] = lkk
        L[k + 1:, k] = A[k + 1:, k] / lkk
        at_k = (a[k] - s[k]) / lkk
        bt_k = (b[k] - s[k]) / lkk
        y[k] = float(special.trunc_mean(at_k, bt_k))
        log_p += float(q[i - k])
        s[k + 1:] += L[k + 1:, k] * y[k]
        A[k + 1:, k + 1:] -= np.outer(L[k + 1:, k], L[k + 1:, k])
    return UCResult(order, L, y, log_p)


def aca(A: np.ndarray, tol: float, max_rank: int):
    """Adaptive cross approximation with full pivoting: A ~ U V^T, max|A - U V^T| <= tol.

    Returns (U, V, capped) with U (rows x k), V (cols x k); capped is True when
    the rank cap stopped the iteration before the tolerance was met.
    """
    R = np.array(A, dtype=np.float64, copy=True)
    us, vs = [], []
    capped = False
    while True:
        if R.size == 0:
            break
        idx = int(np.argmax(np.abs(R)))
        i, j = divmod(idx, R.shape[1])
        piv = R[i, j]
        if abs(piv) <= tol:
            break
        if len(us) >= max_rank:
            capped = True
            break
        u = R[:, j].copy()
        v = R[i, :] / piv
        R -= np.outer(u, v)
        nu_, nv_ = np.linalg.norm(u), np.linalg.norm(v)
        f = np.sqrt(nv_ / nu_)
        us.append(u * f)
        vs.append(v / f)
    if us:
        return np.stack(us, axis=1), np.stack(vs, axis=1), capped
    return np.zeros((A.shape[0], 0)), np.zeros((A.shape[1], 0)), capped


@dataclass
class TLRFactor:
    """L = tile-low-rank Cholesky factor of Sigma[perm][:, perm].

    tile_off[t] .. tile_off[t+1] are the positions of tile t.  B[t] is the dense
    lower diagonal tile, U[(i, j)] (m_i x k) and V[(i, j)] (m_j x k) give
    L_ij ~ U V^T for i > j.
    """
    n: int
    m: int
    perm: np.ndarray
    tile_off: np.ndarray
    B: list
    U: dict = field(default_factory=dict)
    V: dict = field(default_factory=dict)
    capped_tiles: int = 0

    @property
    def r(self) -> int:
        return len(self.B)

    def rank(self, i: int, j: int) -> int:
        return self.U[(i, j)].shape[1]

    def dense(self) -> np.ndarray:
        """Assemble the dense n x n lower factor (for checks at small n)."""
        L = np.zeros((self.n, self.n))
        o = self.tile_off
        for t in range(self.r):
            L[o[t]:o[t + 1], o[t]:o[t + 1]] = self.B[t]
        for (i, j), U in self.U.items():
            L[o[i]:o[i + 1], o[j]:o[j + 1]] = U @ self.V[(i, j)].T
        return L


def tlr_factor(Sigma: np.ndarray, geo_perm: np.ndarray, tile_sizes, a, b, tol: float, max_rank: int,
               reorder: int = REORDER_RBODR) -> TLRFactor:
    """Block-reordered TLR Cholesky factor of a dense covariance (original index order).

    geo_perm / tile_sizes: the geometric indexing (positions -> original indices)
    and its cluster sizes.  a, b: integration limits in original index order
    (used only to choose the order).  reorder: none / Algorithm 4 / Algorithm 5.
    """
    Sigma = np.asarray(Sigma, dtype=np.float64)
    n = Sigma.shape[0]
    offs = np.concatenate([[0], np.cumsum(tile_sizes)])
    blocks = [np.asarray(geo_perm[offs[t]:offs[t + 1]], dtype=np.int64) for t in range(len(tile_sizes))]
    r = len(blocks)
    acur = np.array(a, dtype=np.float64, copy=True)
    bcur = np.array(b, dtype=np.float64, copy=True)
    S = Sigma.copy()                       # Schur complement, original index space

    if reorder == REORDER_BODR:            # Algorithm 4: one estimate per block, then sort
        res = [univariate_conditioning(S[np.ix_(bl, bl)], acur[bl], bcur[bl]) for bl in blocks]
        p = np.array([rs.log_p for rs in res])
        seq = list(range(r))
        for j in range(r):                 # selection sort, first minimum wins
            jt = j + int(np.argmin(p[seq[j:]]))
            seq[j], seq[jt] = seq[jt], seq[j]
        blocks = [blocks[t][res[t].order] for t in seq]

    B, U, V = [], {}, {}
    capped = 0
    for j in range(r):
        yj = None
        if reorder == REORDER_RBODR:       # Algorithm 5, lines 4-9
            res = [univariate_conditioning(S[np.ix_(blocks[l], blocks[l])], acur[blocks[l]], bcur[blocks[l]])
                   for l in range(j, r)]
            jt = j + int(np.argmin([rs.log_p for rs in res]))
            chosen = res[jt - j]
            blocks[j], blocks[jt] = blocks[jt], blocks[j]
            blocks[j] = blocks[j][chosen.order]
            for k in range(j):             # the finished factor rows move with their block
                U[(j, k)], U[(jt, k)] = U[(jt, k)], U[(j, k)]
                V[(j, k)], V[(jt, k)] = V[(jt, k)], V[(j, k)]
                U[(j, k)] = U[(j, k)][chosen.order]
            yj = chosen.y
        bj = blocks[j]
        Ljj = np.linalg.cholesky(S[np.ix_(bj, bj)])          # line 10
        B.append(Ljj)
        cols = []
        for i in range(j + 1, r):                            # lines 11-14
            bi = blocks[i]
            Lij = solve_triangular(Ljj, S[np.ix_(bi, bj)].T, lower=True).T
            Ui, Vi, cap = aca(Lij, tol, max_rank)
            capped += int(cap)
            U[(i, j)], V[(i, j)] = Ui, Vi
            if yj is not None:
                shift = Ui @ (Vi.T @ yj)
                acur[bi] -= shift
                bcur[bi] -= shift
            cols.append(Ui @ Vi.T)
        if j + 1 < r:                                        # lines 15-19, exact Schur update
            rest = np.concatenate(blocks[j + 1:])
            C = np.concatenate(cols, axis=0)
            S[np.ix_(rest, rest)] -= C @ C.T
    perm = np.concatenate(blocks)
    sizes = np.array([bl.size for bl in blocks], dtype=np.int64)
    tile_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return TLRFactor(n, int(max(tile_sizes)) if len(tile_sizes) else 0, perm, tile_off, B, U, V, capped)


class _TileStore:
    """Low-rank tiles of a symmetric TLR matrix keyed by the unordered pair of
    clusters {p, q}: Sigma_pq ~ U V^T with U on p's variables, Sigma_qp = V U^T."""

    def __init__(self):
        self.t = {}

    def get(self, p: int, q: int):
        if (p, q) in self.t:
            return self.t[(p, q)]
        U, V = self.t[(q, p)]
        return V, U

    def set(self, p: int, q: int, U, V):
        self.t.pop((q, p), None)
        self.t[(p, q)] = (U, V)

    def permute(self, c: int, order):
        """Reorder cluster c's variables in every tile that involves it."""
        for key in list(self.t):
            U, V = self.t[key]
            if key[0] == c:
                self.t[key] = (U[order], V)
            elif key[1] == c:
                self.t[key] = (U, V[order])


def tlr_factor_truncated(Sigma: np.ndarray, geo_perm: np.ndarray, tile_sizes, a, b, tol: float, max_rank: int,
                         reorder: int = REORDER_RBODR) -> TLRFactor:
    """Block-reordered TLR Cholesky factor in tile-low-rank arithmetic, Section 3.3 as printed.

    Differs from tlr_factor only in where truncation happens.  Before the
    factorisation the covariance is built as a TLR matrix: dense diagonal
    blocks, every off-diagonal block Sigma_pq compressed by ACA at tol.  The
    loop over positions j is Algorithm 5's (without lines 4-9 for the other
    reorderings):

    * (Algorithm 5) univariate conditioning of every remaining diagonal block
      on its current Schur complement and conditioned limits; the smallest
      estimate takes position j and its pivot order becomes the block's
      within-block order (which reorders that cluster's rows in every tile);
    * Sigma_jj = Cholesky(Sigma_jj);
    * Sigma_ij = Sigma_ij (.) Sigma_jj^-T for i > j: with Sigma_ij = U V^T this
      is U (L_jj^-1 V)^T, then truncated by ACA at tol;
    * (Algorithm 5) a_i, b_i -= Sigma_ij (.) y_j;
    * Sigma_i1j1 = Sigma_i1j1 (-) Sigma_i1j (.) Sigma_j1j^T for j < j1 < i1: the
      low-rank difference U V^T - U_i1j (V_i1j^T V_j1j) U_j1j^T truncated by
      ACA at tol; the diagonal blocks (i1 = j1) are dense and updated exactly.

    Readings where the paper is silent (restated in the design notes):
    * truncation = the full-pivoting ACA of aca() on the tile written out
      densely, the same rule as the covariance construction;
    * a product with a rank-0 factor is zero: the tile it would update is left
      as it is (not re-truncated);
    * capped_tiles counts every truncation the rank cap stopped (construction,
      (.) and (-) alike).
    """
    Sigma = np.asarray(Sigma, dtype=np.float64)
    n = Sigma.shape[0]
    offs = np.concatenate([[0], np.cumsum(tile_sizes)])
    idx = [np.asarray(geo_perm[offs[t]:offs[t + 1]], dtype=np.int64) for t in range(len(tile_sizes))]
    r = len(idx)
    acur = np.array(a, dtype=np.float64, copy=True)
    bcur = np.array(b, dtype=np.float64, copy=True)
    pos = list(range(r))                   # pos[j] = cluster at position j
    capped = 0

    if reorder == REORDER_BODR:            # Algorithm 4 on the covariance itself
        res = [univariate_conditioning(Sigma[np.ix_(bl, bl)], acur[bl], bcur[bl]) for bl in idx]
        p = np.array([rs.log_p for rs in res])
        for j in range(r):
            jt = j + int(np.argmin(p[pos[j:]]))
            pos[j], pos[jt] = pos[jt], pos[j]
        idx = [idx[c][res[c].order] for c in range(r)]

    # the TLR covariance: dense diagonal blocks, ACA-compressed off-diagonal blocks
    D = [Sigma[np.ix_(bl, bl)].copy() for bl in idx]
    T = _TileStore()
    for p_ in range(r):
        for q_ in range(p_ + 1, r):
            U, V, cp = aca(Sigma[np.ix_(idx[p_], idx[q_])], tol, max_rank)
            capped += int(cp)
            T.set(p_, q_, U, V)

    B = []
    for j in range(r):
        yj = None
        if reorder == REORDER_RBODR:       # Algorithm 5, lines 4-8
            res = [univariate_conditioning(D[pos[l]], acur[idx[pos[l]]], bcur[idx[pos[l]]]) for l in range(j, r)]
            jt = j + int(np.argmin([rs.log_p for rs in res]))
            chosen = res[jt - j]
            pos[j], pos[jt] = pos[jt], pos[j]
            c = pos[j]
            o = chosen.order
            idx[c] = idx[c][o]
            D[c] = D[c][np.ix_(o, o)]
            T.permute(c, o)
            yj = chosen.y
        cj = pos[j]
        Ljj = np.linalg.cholesky(D[cj])                      # line 10
        B.append(Ljj)
        for i in range(j + 1, r):                            # lines 11-14
            ci = pos[i]
            U, V = T.get(ci, cj)
            if U.shape[1]:
                U, V, cp = aca(U @ solve_triangular(Ljj, V, lower=True).T, tol, max_rank)
                capped += int(cp)
            T.set(ci, cj, U, V)
            if yj is not None and U.shape[1]:
                shift = U @ (V.T @ yj)
                acur[idx[ci]] -= shift
                bcur[idx[ci]] -= shift
        for j1 in range(j + 1, r):                           # lines 15-19
            U1, V1 = T.get(pos[j1], cj)
            if not U1.shape[1]:
                continue
            for i1 in range(j1, r):
                U2, V2 = T.get(pos[i1], cj)
                if not U2.shape[1]:
                    continue
                prod = U2 @ (V2.T @ V1) @ U1.T               # Sigma_i1j Sigma_j1j^T
                if i1 == j1:
                    D[pos[i1]] -= prod
                else:
                    Us, Vs = T.get(pos[i1], pos[j1])
                    U, V, cp = aca(Us @ Vs.T - prod, tol, max_rank)
                    capped += int(cp)
                    T.set(pos[i1], pos[j1], U, V)
    perm = np.concatenate([idx[c] for c in pos])
    sizes = np.array([idx[c].size for c in pos], dtype=np.int64)
    tile_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    U, V = {}, {}
    for i in range(r):
        for j in range(i):
            U[(i, j)], V[(i, j)] = T.get(pos[i], pos[j])
    return TLRFactor(n, int(max(tile_sizes)) if len(tile_sizes) else 0, perm, tile_off, B, U, V, capped)


def reorder_within_tiles(F: TLRFactor, a, b) -> TLRFactor:
    """Post-hoc within-tile reordering of a finished factor for new limits.

    Not in the paper; derived from its factor structure:
    the block reorderings of Section 3.3 also reorder variables within each
    diagonal block, and that within-block order depends on the limits, which a
    resident factor meets anew in every request.  For each tile j:

    * P_j: the pivot order of univariate conditioning on the tile's conditional
      covariance given all earlier tiles, B_j B_j^T (the Schur complement of the
      tile), with the new limits of its variables (not shifted by earlier tiles);
    * the new diagonal block is Lt_j = chol(P_j B_j B_j^T P_j^T), and
      Q_j = B_j^-1 P_j^T Lt_j is orthogonal (Q_j Q_j^T = B_j^-1 P_j^T Lt_j Lt_j^T
      P_j B_j^-T = I);
    * the factor L' = diag(P) L diag(Q) is lower block triangular with diagonal
      blocks P_j B_j Q_j = Lt_j and L' L'^T = P L L^T P^T: it is the TLR factor of
      the reordered variables.  Its off-diagonal tiles keep their ranks: the rows
      of tile j in row blocks are permuted (U_jk -> P_j U_jk) and its column blocks
      rotated (V_ij -> Q_j^T V_ij).

    a, b: new limits in original index order.  Returns a new TLRFactor.
    """
    a = np.asarray(a, dtype=np.float64)[F.perm]
    b = np.asarray(b, dtype=np.float64)[F.perm]
    o = F.tile_off
    perm = F.perm.copy()
    B, U, V = list(F.B), dict(F.U), dict(F.V)
    for j in range(F.r):
        S = F.B[j] @ F.B[j].T
        uc = univariate_conditioning(S, a[o[j]:o[j + 1]], b[o[j]:o[j + 1]])
        p = uc.order
        Lt = np.linalg.cholesky(S[np.ix_(p, p)])
        Pt_Lt = np.zeros_like(Lt)
        Pt_Lt[p, :] = Lt                      # P_j^T Lt_j (P_j picks rows p)
        Q = solve_triangular(F.B[j], Pt_Lt, lower=True)
        B[j] = Lt
        perm[o[j]:o[j + 1]] = F.perm[o[j]:o[j + 1]][p]
        for k in range(j):                    # rows of tile j in the row blocks to its left
            U[(j, k)] = F.U[(j, k)][p]
        for i in range(j + 1, F.r):           # column blocks below tile j
            V[(i, j)] = Q.T @ F.V[(i, j)]
    return TLRFactor(F.n, F.m, perm, F.tile_off.copy(), B, U, V, F.capped_tiles)
