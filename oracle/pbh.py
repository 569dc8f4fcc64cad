"""Path-based Hessian bound (Thm. 1) and its baselines, plain FP64.

Steps, in the paper's order (Sec. IV-A):

1. Tube set -> box X (Eq. 18a box ``c + diag(sigma) E``, or a zonotope ``c + G E`` reduced to its interval
   hull ``c +- ||G||_{1,r}`` with the row-wise l1 norm of Sec. III and Eq. 21), hulled with the nominal
   point so that ``alpha~ in X`` as Thm. 1 requires.
2. Displacement set Delta = X (-) alpha~ (Eq. 12).
3. For each output row l and each structurally nonzero Hessian entry (j <= k):
   evaluate [H_{l,kj}] over the prefix set X^(j) (coordinates 0..j range over X, the rest are fixed at
   the nominal; Sec. IV-A, "coordinate-wise path"), multiply by Delta_j * Delta_k (j < k) or by
   1/2 Delta_k^2 (j = k, the interval of squares), and sum the terms one by one (Eq. 15).

``ih_expand`` (Eq. 13) evaluates every entry over the full X; ``ih_classic`` (Eq. 12) forms the interval
quadratic form 1/2 Delta^T ([H](X) Delta). ``gamma_map`` is the zonotope map of Sec. IV-C.
"""
from __future__ import annotations

import numpy as np

from .dynamics import iv_add, iv_mul, iv_scale, iv_sqr


def box_from_set(nominal: np.ndarray, radii=None, G=None, center=None):
    """Interval hull of the tube set, hulled with the nominal point. Returns (lo, hi) FP64 [n]."""
    a = np.asarray(nominal, np.float64)
    c = a if center is None else np.asarray(center, np.float64)
    if G is not None:
        half = np.abs(np.asarray(G, np.float64)).sum(axis=1)      # ||G||_{1,r}
    else:
        half = np.asarray(radii, np.float64)
    lo = np.minimum(c - half, a)
    hi = np.maximum(c + half, a)
    return lo, hi


def prefix_box(lo: np.ndarray, hi: np.ndarray, nominal: np.ndarray, j: int):
    """X^(j): coordinates 0..j range over [lo, hi], coordinates > j are fixed at the nominal."""
    plo = np.array(nominal, np.float64)
    phi = np.array(nominal, np.float64)
    plo[: j + 1] = lo[: j + 1]
    phi[: j + 1] = hi[: j + 1]
    return plo, phi


def ordered_prefix_box(lo, hi, nominal, rank, j: int):
    """X^(j) for the path order with ranks ``rank`` (rank[c] = position of coordinate c on the path):
    the coordinates at or before j range over [lo, hi], the later ones sit at the nominal."""
    inpre = np.asarray(rank) <= rank[j]
    a = np.asarray(nominal, np.float64)
    return np.where(inpre, lo, a), np.where(inpre, hi, a)


def pbh(dyn, nominal: np.ndarray, lo: np.ndarray, hi: np.ndarray, order=None):
    """Thm. 1 enclosure [R_lo, R_hi] of the linearization error of every output row. ``order``: the path
    order as a permutation of the coordinates (default the natural one); each entry (j, k) is evaluated
    over the prefix set of whichever of j, k comes first on the path."""
    a = np.asarray(nominal, np.float64)
    D = [(lo[i] - a[i], hi[i] - a[i]) for i in range(dyn.n)]
    R_lo = np.zeros(dyn.n_x)
    R_hi = np.zeros(dyn.n_x)
    rank = None
    if order is not None:
        rank = np.empty(dyn.n, int)
        rank[np.asarray(order)] = np.arange(dyn.n)
    for row in range(dyn.n_x):
        R = (0.0, 0.0)
        for j, k, fn in dyn.hessian_terms(row):
            if rank is None:
                plo, phi = prefix_box(lo, hi, a, min(j, k))
            else:
                plo, phi = ordered_prefix_box(lo, hi, a, rank, j if rank[j] <= rank[k] else k)
            Hv = fn(plo, phi)
            if j == k:
                term = iv_scale(0.5, iv_mul(Hv, iv_sqr(D[k])))
            else:
                term = iv_mul(Hv, iv_mul(D[j], D[k]))
            R = iv_add(R, term)
        R_lo[row], R_hi[row] = R
    return R_lo, R_hi


def ih_expand(dyn, nominal, lo, hi):
    """Eq. 13: the same expansion with every Hessian entry over the full box X."""
    a = np.asarray(nominal, np.float64)
    D = [(lo[i] - a[i], hi[i] - a[i]) for i in range(dyn.n)]
    R_lo = np.zeros(dyn.n_x)
    R_hi = np.zeros(dyn.n_x)
    for row in range(dyn.n_x):
        R = (0.0, 0.0)
        for j, k, fn in dyn.hessian_terms(row):
            Hv = fn(lo, hi)
            if j == k:
                term = iv_scale(0.5, iv_mul(Hv, iv_sqr(D[k])))
            else:
                term = iv_mul(Hv, iv_mul(D[j], D[k]))
            R = iv_add(R, term)
        R_lo[row], R_hi[row] = R
    return R_lo, R_hi


def ih_classic(dyn, nominal, lo, hi):
    """Eq. 12: 1/2 Delta^T ([H](X) Delta) with interval matrix-vector then interval dot products."""
    a = np.asarray(nominal, np.float64)
    D = [(lo[i] - a[i], hi[i] - a[i]) for i in range(dyn.n)]
    R_lo = np.zeros(dyn.n_x)
    R_hi = np.zeros(dyn.n_x)
    for row in range(dyn.n_x):
        Hfull = {}
        for j, k, fn in dyn.hessian_terms(row):
            Hv = fn(lo, hi)
            Hfull[(j, k)] = Hv
            Hfull[(k, j)] = Hv
        idx = sorted({p for jk in Hfull for p in jk})
        R = (0.0, 0.0)
        for p in idx:
            v = (0.0, 0.0)
            for q in idx:
                if (p, q) in Hfull:
                    v = iv_add(v, iv_mul(Hfull[(p, q)], D[q]))
            R = iv_add(R, iv_mul(D[p], v))
        R_lo[row], R_hi[row] = iv_scale(0.5, R)
    return R_lo, R_hi


def gamma_map(r_lo: np.ndarray, r_hi: np.ndarray, pad: float = 0.0):
    """Zonotope of an interval bound (Sec. IV-C): c = (lo+hi)/2, R = diag((hi-lo)/2) (+ diagonal padding)."""
    c = 0.5 * (np.asarray(r_lo, np.float64) + np.asarray(r_hi, np.float64))
    rad = 0.5 * (np.asarray(r_hi, np.float64) - np.asarray(r_lo, np.float64)) + pad
    return c, rad


def pbh_workload_row(dyn, nominal, radii=None, G=None, center=None):
    """Convenience: set -> box -> Thm. 1 for one timestep. Returns (R_lo, R_hi, J, lo, hi)."""
    lo, hi = box_from_set(nominal, radii=radii, G=G, center=center)
    R_lo, R_hi = pbh(dyn, nominal, lo, hi)
    return R_lo, R_hi, dyn.jacobian(nominal), lo, hi


def split_pieces(nominal: np.ndarray, lo: np.ndarray, hi: np.ndarray, dims):
    """Input-domain partitioning (Sec. IV-D): the box cut at the nominal along each coordinate of
    ``dims`` into its lower part [lo_j, a_j] and upper part [a_j, hi_j]; 2^len(dims) pieces, each still
    containing the nominal (Thm. 1). Yields (lo_p, hi_p) in the order of the bits of p (bit i = upper part
    of dims[i])."""
    a = np.asarray(nominal, np.float64)
    for p in range(1 << len(dims)):
        lp, hp = np.array(lo, np.float64), np.array(hi, np.float64)
        for i, j in enumerate(dims):
            if (p >> i) & 1:
                lp[j] = a[j]
            else:
                hp[j] = a[j]
        yield lp, hp


def pbh_partitioned(dyn, nominal, lo, hi, dims):
    """Thm. 1 on every piece of the partition, and the componentwise hull of the pieces' bounds: a bound
    of the remainder over the whole box (every point lies in some piece)."""
    R_lo, R_hi = None, None
    for lp, hp in split_pieces(nominal, lo, hi, dims):
        l, h = pbh(dyn, nominal, lp, hp)
        R_lo = l if R_lo is None else np.minimum(R_lo, l)
        R_hi = h if R_hi is None else np.maximum(R_hi, h)
    return R_lo, R_hi


def recentred_cuts(lo_j: float, hi_j: float, K: int):
    """The K equal pieces of [lo_j, hi_j] and their midpoints, with the interior cut points and the
    midpoints as the library forms them in FP32 from FP32 ends (round to nearest: w = hi - lo,
    p_k = lo + w (k / K), beta_k = p_k / 2 + p_{k+1} / 2): they are part of the partition's definition, so
    both sides use the same points. The outer cuts are the box ends themselves (so the pieces cover the
    box whatever its ends are), and each midpoint is kept inside its piece. Returns FP64 arrays (cuts
    [K + 1], mids [K])."""
    f = np.float32
    lo32, hi32 = f(lo_j), f(hi_j)
    w = f(hi32 - lo32)
    c32 = [lo32]
    for k in range(1, K):
        p = f(lo32 + f(w * f(f(k) / f(K))))
        c32.append(min(max(p, lo32), hi32))
    c32.append(hi32)
    cuts = np.array([float(lo_j)] + [float(c) for c in c32[1:K]] + [float(hi_j)], np.float64)
    mids = np.array([f(f(f(0.5) * c32[k]) + f(f(0.5) * c32[k + 1])) for k in range(K)], np.float64)
    mids = np.minimum(np.maximum(mids, cuts[:-1]), cuts[1:])
    return cuts, mids


def pbh_recentred(dyn, nominal, lo, hi, dims, K: int, A=None):
    """Input-domain partitioning with re-centred pieces (Sec. IV-D names partitioning; Thm. 1 needs the
    expansion point inside the set, so a piece away from the nominal is expanded around a point beta of its
    own). For alpha in a piece P with beta in P, and A the returned linearization (default the Jacobian at
    the nominal),
        r(alpha; alpha~) = f(alpha) - f(alpha~) - A (alpha - alpha~)
                         = [f(alpha) - f(beta) - J(beta)(alpha - beta)]     Thm. 1 around beta over P
                         + [f(beta) - f(alpha~) - A (beta - alpha~)]       a point value
                         + (J(beta) - A)(alpha - beta)                      an interval product over P.
    Each coordinate d of ``dims`` is cut alone into K equal pieces (``recentred_cuts``; the other
    coordinates keep their whole range, beta = the nominal with beta_d = the piece's midpoint); the hull
    over the pieces bounds the remainder over the box. The plain bound w.r.t. A (Thm. 1 plus the
    interval product (J - A) Delta) and the bounds of the several coordinates are intersected (each is
    valid), so the result is never wider than the plain one. FP64 numpy (R_lo, R_hi)."""
    a = np.asarray(nominal, np.float64)
    A = dyn.jacobian(a) if A is None else np.asarray(A, np.float64)
    f0 = dyn.f(a)
    R_lo, R_hi = pbh(dyn, a, lo, hi)
    M0 = dyn.jacobian(a) - A
    D0l, D0h = np.asarray(lo, np.float64) - a, np.asarray(hi, np.float64) - a
    R_lo = R_lo + np.minimum(M0 * D0l, M0 * D0h).sum(axis=1)
    R_hi = R_hi + np.maximum(M0 * D0l, M0 * D0h).sum(axis=1)
    for d in dims:
        cuts, mids = recentred_cuts(lo[d], hi[d], K)
        H_lo = np.full(dyn.n_x, np.inf)
        H_hi = np.full(dyn.n_x, -np.inf)
        for k in range(K):
            lp, hp = np.array(lo, np.float64), np.array(hi, np.float64)
            lp[d], hp[d] = cuts[k], cuts[k + 1]
            beta = a.copy()
            beta[d] = mids[k]
            l, h = pbh(dyn, beta, lp, hp)
            point = dyn.f(beta) - f0 - A @ (beta - a)
            M = dyn.jacobian(beta) - A
            Dl, Dh = lp - beta, hp - beta
            cl = np.minimum(M * Dl, M * Dh).sum(axis=1)
            ch = np.maximum(M * Dl, M * Dh).sum(axis=1)
            H_lo = np.minimum(H_lo, l + point + cl)
            H_hi = np.maximum(H_hi, h + point + ch)
        R_lo = np.maximum(R_lo, H_lo)
        R_hi = np.minimum(R_hi, H_hi)
    return R_lo, R_hi
