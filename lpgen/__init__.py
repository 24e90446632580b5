"""Seeded synthetic LP generators shared by the tests, the benchmark and the oracle.

This module builds problem data only.  It holds none of the solver's arithmetic
(no PDHG step, no KKT evaluation, no scaling); it draws random numbers and
assembles LPs in the form of the paper's Eq. (LP):

    min c^T x   s.t.  A x = b,  G x >= h,  l <= x <= u,
    K = [A; G] (equality rows first), q = [b; h], m1 = rows of A.

Every generator returns a dict with

    m, n, m1            : int
    row_ptr (int64, m+1), col_idx (int32, nnz), val (float64, nnz)   -- K in CSR
    c, q, l, u          : float64 arrays (l/u use -inf/+inf for absent bounds)

and, for the planted-optimum families, the planted optimum ``x_star``,
``y_star``, ``lam_star`` and its objective ``obj_star``.

Planted optimum.  (x*, y*, lambda*) is drawn first with complementarity built in:
lambda*_j > 0 only where x*_j sits at a finite lower bound, < 0 only where it sits
at a finite upper bound, y*_i > 0 only on inequality rows that are tight.  Then
b = A x*, h = G x* (minus a positive slack on the non-tight inequality rows) and
c = K^T y* + lambda*.  The primal and dual objectives coincide by construction,
so x*, y* is optimal for the generated LP.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "csr_from_coo",
    "planted_from_structure",
    "planted_small",
    "planted_random",
    "batch_planted",
    "mcf",
    "transport_family",
    "transport_instance",
    "planted_zipf",
    "box_only",
    "tiny_lp",
    "random_csr",
]


def csr_from_coo(m, n, rows, cols, vals):
    """Sort (row, col) pairs into CSR, summing nothing: duplicate pairs are dropped
    (the first occurrence in sorted order is kept)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    key = rows * np.int64(n) + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    keep = np.ones(key.shape[0], dtype=bool)
    if key.shape[0] > 1:
        keep[1:] = key[1:] != key[:-1]
    key = key[keep]
    vals = vals[order][keep]
    r = key // n
    ccol = (key % n).astype(np.int32)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=m), out=row_ptr[1:])
    return row_ptr, ccol, vals


def _csr_matvec(row_ptr, col_idx, val, x):
    """y = K x for problem assembly (b, h from x*)."""
    m = row_ptr.shape[0] - 1
    prod = val * x[col_idx]
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(row_ptr))
    return np.bincount(rows, weights=prod, minlength=m)


def _csr_rmatvec(row_ptr, col_idx, val, y, n):
    """g = K^T y for problem assembly (c from y*)."""
    m = row_ptr.shape[0] - 1
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(row_ptr))
    return np.bincount(col_idx, weights=val * y[rows], minlength=n)


def planted_from_structure(rng, m, n, m1, row_ptr, col_idx, val, bound_class,
                           box_u, frac_active=0.5):
    """Plant an optimum on a given sparsity structure.

    bound_class[j] in {0: free, 1: box [0, box_u[j]], 2: lower-bounded [0, inf)}.
    Box columns are split in thirds (at lower / at upper / interior); lower-bounded
    columns in halves (at lower / interior).  Inequality rows are tight with
    probability ``frac_active`` (y* = |N(0,1)|), otherwise slack (y* = 0).
    """
    x = np.zeros(n)
    lam = np.zeros(n)
    l = np.full(n, -np.inf)
    u = np.full(n, np.inf)
    free = bound_class == 0
    box = bound_class == 1
    low = bound_class == 2
    x[free] = rng.uniform(-10.0, 10.0, free.sum())
    # box columns
    jb = np.flatnonzero(box)
    l[jb] = 0.0
    u[jb] = box_u[jb]
    sub = rng.integers(0, 3, jb.shape[0])
    at_l, at_u, inner = jb[sub == 0], jb[sub == 1], jb[sub == 2]
    x[at_l] = 0.0
    lam[at_l] = np.abs(rng.standard_normal(at_l.shape[0]))
    x[at_u] = u[at_u]
    lam[at_u] = -np.abs(rng.standard_normal(at_u.shape[0]))
    x[inner] = u[inner] * rng.uniform(0.1, 0.9, inner.shape[0])
    # lower-bounded columns
    jl = np.flatnonzero(low)
    l[jl] = 0.0
    sub = rng.integers(0, 2, jl.shape[0])
    x[jl[sub == 0]] = 0.0
    lam[jl[sub == 0]] = np.abs(rng.standard_normal((sub == 0).sum()))
    x[jl[sub == 1]] = rng.uniform(1.0, 10.0, (sub == 1).sum())
    # duals of the rows
    y = np.zeros(m)
    y[:m1] = rng.standard_normal(m1)
    m2 = m - m1
    active = rng.random(m2) < frac_active
    y[m1:][active] = np.abs(rng.standard_normal(active.sum()))
    Kx = _csr_matvec(row_ptr, col_idx, val, x)
    q = Kx.copy()
    slack = np.abs(rng.standard_normal(m2))
    q[m1:][~active] -= slack[~active]
    c = _csr_rmatvec(row_ptr, col_idx, val, y, n) + lam
    return dict(m=m, n=n, m1=m1, row_ptr=row_ptr, col_idx=col_idx, val=val,
                c=c, q=q, l=l, u=u, x_star=x, y_star=y, lam_star=lam,
                obj_star=float(c @ x))


def planted_random(rng, m1, m2, n, nnz, box_u=10.0):
    """A planted-optimum LP with ``nnz`` distinct positions drawn uniformly without
    replacement and N(0,1) values.  Columns (random permutation): a quarter at l=0
    (bounds [0, box_u], lambda* > 0), a quarter at u=box_u (lambda* < 0), a quarter
    interior of [0, box_u], the rest free.  Half of the inequality rows are tight."""
    m = m1 + m2
    nnz = min(int(nnz), m * n)
    pos = rng.choice(m * n, size=nnz, replace=False) if m > 0 else np.zeros(0, dtype=np.int64)
    rows, cols = pos // n, pos % n
    vals = rng.standard_normal(nnz)
    row_ptr, col_idx, val = csr_from_coo(m, n, rows, cols, vals)
    perm = rng.permutation(n)
    q4 = n // 4
    x = np.zeros(n)
    lam = np.zeros(n)
    l = np.zeros(n)
    u = np.full(n, box_u)
    at_l, at_u, inner, free = perm[:q4], perm[q4:2 * q4], perm[2 * q4:3 * q4], perm[3 * q4:]
    lam[at_l] = np.abs(rng.standard_normal(at_l.shape[0]))
    x[at_u] = box_u
    lam[at_u] = -np.abs(rng.standard_normal(at_u.shape[0]))
    x[inner] = rng.uniform(0.1 * box_u, 0.9 * box_u, inner.shape[0])
    l[free] = -np.inf
    u[free] = np.inf
    x[free] = rng.uniform(-box_u, box_u, free.shape[0])
    y = np.zeros(m)
    y[:m1] = rng.standard_normal(m1)
    act = rng.permutation(m2)[: m2 // 2]
    y[m1 + act] = np.abs(rng.standard_normal(act.shape[0]))
    Kx = _csr_matvec(row_ptr, col_idx, val, x)
    q = Kx.copy()
    slack_rows = np.setdiff1d(np.arange(m2), act)
    q[m1 + slack_rows] -= np.abs(rng.standard_normal(slack_rows.shape[0]))
    c = _csr_rmatvec(row_ptr, col_idx, val, y, n) + lam
    return dict(m=m, n=n, m1=m1, row_ptr=row_ptr, col_idx=col_idx, val=val,
                c=c, q=q, l=l, u=u, x_star=x, y_star=y, lam_star=lam,
                obj_star=float(c @ x))


def planted_small(seed=0, m1=200, m2=300, n=1000, nnz=5000):
    """The small planted-optimum LP: m1 equality rows, m2 inequality rows, n columns,
    exactly ``nnz`` distinct positions (see ``planted_random``)."""
    return planted_random(np.random.default_rng(seed), m1, m2, n, nnz)


def batch_planted(count, seed=0, n_lo=50, n_hi=5000, m_ratio=(0.3, 0.8), density=(0.005, 0.05),
                  eq_frac=0.4):
    """The batched workload: ``count`` independent planted LPs, LP i drawn with seed
    ``seed + i``: n ~ U(n_lo, n_hi) (integer), m = round(U(m_ratio) n), m1 = round(eq_frac m),
    density ~ U(density) of the m x n positions, values N(0,1), bounds as planted_random."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed + i)
        n = int(rng.integers(n_lo, n_hi + 1))
        m = int(round(rng.uniform(*m_ratio) * n))
        m1 = int(round(eq_frac * m))
        d = rng.uniform(*density)
        nnz = max(1, int(round(d * m * n))) if m > 0 else 0
        out.append(planted_random(rng, m1, m - m1, n, nnz))
    return out


def _zipf_lengths(rng, m, target_nnz, n, a=1.5, cap=10000):
    """Row lengths: k ~ Zipf(a) truncated at ``cap`` (rejection), then
    L = ceil(s k) with s found by bisection so that sum(L) ~= target_nnz."""
    k = np.empty(0, dtype=np.int64)
    while k.shape[0] < m:
        d = rng.zipf(a, size=2 * m)
        k = np.concatenate([k, d[d <= cap]])
    k = k[:m].astype(np.float64)
    lo, hi = 0.0, float(target_nnz) / m + 1.0
    for _ in range(100):
        s = 0.5 * (lo + hi)
        tot = np.ceil(s * k).sum()
        if tot > target_nnz:
            hi = s
        else:
            lo = s
    L = np.ceil(lo * k).astype(np.int64)
    return np.minimum(L, n)


def planted_zipf(seed=0, n=2_000_000, m=1_000_000, eq_frac=0.4, nnz=20_000_000,
                 zipf_a=1.5, zipf_cap=10000):
    """The large sparse planted LP: m rows (``eq_frac`` equalities), n columns,
    Zipf(1.5) row lengths (truncated at 1e4, then scaled so the total is ~nnz),
    columns uniform without repeats inside a row, values +-10^U(-3,3).
    Bounds: 25% free, 50% [0, u] with u ~ U(1, 100), 25% [0, inf).
    Optimum planted per bound class (see ``planted_from_structure``).
    Smaller instances of the same recipe come from shrinking n, m and nnz together.
    """
    rng = np.random.default_rng(seed)
    m1 = int(round(eq_frac * m))
    L = _zipf_lengths(rng, m, nnz, n, zipf_a, zipf_cap)
    rows = np.repeat(np.arange(m, dtype=np.int64), L)
    cols = rng.integers(0, n, rows.shape[0])
    tot = rows.shape[0]
    mag = 10.0 ** rng.uniform(-3.0, 3.0, tot)
    sign = np.where(rng.random(tot) < 0.5, -1.0, 1.0)
    row_ptr, col_idx, val = csr_from_coo(m, n, rows, cols, sign * mag)
    del rows, cols, mag, sign
    r = rng.random(n)
    bound_class = np.where(r < 0.25, 0, np.where(r < 0.75, 1, 2)).astype(np.int8)
    box_u = rng.uniform(1.0, 100.0, n)
    return planted_from_structure(rng, m, n, m1, row_ptr, col_idx, val, bound_class, box_u)


def box_only(seed=0, n=64, free_frac=0.0):
    """An LP with no rows (m = 0): min c^T x over a box.  Finite bounds everywhere
    except a ``free_frac`` share of free columns, which get c_j = 0 so that the LP
    stays bounded.  Its optimum is closed-form: x_j = l_j if c_j > 0, u_j if c_j < 0."""
    rng = np.random.default_rng(seed)
    l = rng.uniform(-5.0, 0.0, n)
    u = l + rng.uniform(0.5, 5.0, n)
    c = rng.standard_normal(n)
    free = rng.random(n) < free_frac
    l[free] = -np.inf
    u[free] = np.inf
    c[free] = 0.0
    return dict(m=0, n=n, m1=0, row_ptr=np.zeros(1, dtype=np.int64),
                col_idx=np.zeros(0, dtype=np.int32), val=np.zeros(0),
                c=c, q=np.zeros(0), l=l, u=u)


def tiny_lp(seed=0, n=5, m1=1, m2=2):
    """A tiny dense LP with finite bounds and a feasible interior point, for brute-force
    vertex enumeration: A, G ~ N(0,1), x0 ~ U(l, u), b = A x0, h = G x0 - |N(0,1)|."""
    rng = np.random.default_rng(seed)
    m = m1 + m2
    K = rng.standard_normal((m, n))
    l = rng.uniform(-3.0, -0.5, n)
    u = rng.uniform(0.5, 3.0, n)
    x0 = rng.uniform(0.5 * l, 0.5 * u)
    q = K @ x0
    q[m1:] -= np.abs(rng.standard_normal(m2))
    c = rng.standard_normal(n)
    rows, cols = np.nonzero(np.ones((m, n)))
    row_ptr, col_idx, val = csr_from_coo(m, n, rows, cols, K[rows, cols])
    return dict(m=m, n=n, m1=m1, row_ptr=row_ptr, col_idx=col_idx, val=val,
                c=c, q=q, l=l, u=u, K_dense=K)


def random_csr(seed, m, n, lengths, dist="normal"):
    """A CSR matrix with the given row lengths (distinct uniform columns per row),
    used to exercise SpMV on chosen row-length regimes (empty rows, 1, 31/32/33, long)."""
    rng = np.random.default_rng(seed)
    lengths = np.minimum(np.asarray(lengths, dtype=np.int64), n)
    rows, cols = [], []
    for i, L in enumerate(lengths):
        if L:
            rows.append(np.full(L, i, dtype=np.int64))
            cols.append(rng.choice(n, size=L, replace=False))
    rows = np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64)
    cols = np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64)
    if dist == "normal":
        vals = rng.standard_normal(rows.shape[0])
    else:
        vals = np.where(rng.random(rows.shape[0]) < 0.5, -1.0, 1.0) * 10.0 ** rng.uniform(-3, 3, rows.shape[0])
    return csr_from_coo(m, n, rows, cols, vals)


def mcf(seed=0, nodes=200_000, arcs=1_000_000, commodities=8, walk_len=20, fill=0.5):
    """Multicommodity-flow LP: a random directed graph on ``nodes`` nodes with ``arcs``
    arcs, the first ``nodes`` of which form a random Hamiltonian cycle (so every node
    has an out-arc), and ``commodities`` commodities.  Columns x_{k,a} >= 0 in
    commodity-major order (k * arcs + a), costs U(1, 10).
    Rows: conservation, one equality per (k, v) with +1 on the arcs leaving v and -1 on
    the arcs entering v (m1 = commodities * nodes), then one capacity row per arc,
    -sum_k x_{k,a} >= -cap_a with cap_a ~ U(5, 50).
    A feasible flow is planted: each commodity routes random walks of ``walk_len`` arcs
    with flow U(0.1, 1) each until the commodities together use about ``fill`` of the
    total capacity; b is its net flow, and an arc whose planted load exceeds 90 % of its
    capacity gets capacity load / 0.9 (so the planted flow stays strictly feasible)."""
    rng = np.random.default_rng(seed)
    V, A, Kc = nodes, arcs, commodities
    perm = rng.permutation(V)
    tail = np.empty(A, dtype=np.int64)
    head = np.empty(A, dtype=np.int64)
    tail[:V] = perm
    head[:V] = np.roll(perm, -1)
    t = rng.integers(0, V, A - V)
    h = rng.integers(0, V - 1, A - V)
    h = h + (h >= t)                      # no self-loops
    tail[V:], head[V:] = t, h
    cap = rng.uniform(5.0, 50.0, A)
    cost = rng.uniform(1.0, 10.0, Kc * A)
    # out-arc lists for the random walks
    order = np.argsort(tail, kind="stable")
    out_ptr = np.zeros(V + 1, dtype=np.int64)
    np.cumsum(np.bincount(tail, minlength=V), out=out_ptr[1:])
    out_arcs = order
    walks_per_k = max(1, int(fill * cap.sum() / (Kc * walk_len * 0.55)))
    flow = np.zeros((Kc, A))
    for k in range(Kc):
        cur = rng.integers(0, V, walks_per_k)
        amount = rng.uniform(0.1, 1.0, walks_per_k)
        for _ in range(walk_len):
            deg = out_ptr[cur + 1] - out_ptr[cur]
            pick = out_arcs[out_ptr[cur] + (rng.random(walks_per_k) * deg).astype(np.int64)]
            np.add.at(flow[k], pick, amount)
            cur = head[pick]
    load = flow.sum(axis=0)
    cap = np.maximum(cap, load / 0.9)
    x = flow.reshape(-1)                  # commodity-major, matches the columns
    # conservation rows (k, v): +1 at the tail node, -1 at the head node of each arc
    m1 = Kc * V
    cols = np.arange(Kc * A, dtype=np.int64)
    kk = cols // A
    aa = cols % A
    r_out = kk * V + tail[aa]
    r_in = kk * V + head[aa]
    r_cap = m1 + aa
    rows = np.concatenate([r_out, r_in, r_cap])
    cc = np.concatenate([cols, cols, cols])
    vals = np.concatenate([np.ones(Kc * A), -np.ones(Kc * A), -np.ones(Kc * A)])
    m = m1 + A
    row_ptr, col_idx, val = csr_from_coo(m, Kc * A, rows, cc, vals)
    b = np.bincount(r_out, weights=x, minlength=m1) - np.bincount(r_in, weights=x, minlength=m1)
    q = np.concatenate([b[:m1], -cap])
    n = Kc * A
    return dict(m=m, n=n, m1=m1, row_ptr=row_ptr, col_idx=col_idx, val=val, c=cost, q=q,
                l=np.zeros(n), u=np.full(n, np.inf), x_feasible=x)


def transport_family(supplies=40, demands=60, seed=0):
    """A family of transportation LPs sharing one cost matrix: supply and demand points
    uniform in [0,1]^2, cost = Euclidean distance + N(0, 0.05) (drawn once per family)."""
    rng = np.random.default_rng(seed)
    P = rng.random((supplies, 2))
    Q = rng.random((demands, 2))
    cost = np.sqrt(((P[:, None, :] - Q[None, :, :]) ** 2).sum(-1)) + rng.normal(0.0, 0.05, (supplies, demands))
    return dict(S=supplies, D=demands, cost=cost, seed=seed)


def transport_instance(family, seed):
    """One LP of the family: supplies s ~ Gamma(2, 50), demands d ~ Gamma(2, 50) rescaled
    to the same total; min sum c_ij x_ij  s.t.  sum_j x_ij = s_i, sum_i x_ij = d_j, x >= 0
    (all rows equalities, one of them redundant).  Column i*D + j is x_ij.  ``features``
    holds (s, d), the parameters a warm-start model sees."""
    S, D = family["S"], family["D"]
    rng = np.random.default_rng(seed)
    s = rng.gamma(2.0, 50.0, S)
    d = rng.gamma(2.0, 50.0, D)
    d *= s.sum() / d.sum()
    n, m = S * D, S + D
    cols = np.arange(n, dtype=np.int64)
    rows = np.concatenate([cols // D, S + cols % D])
    row_ptr, col_idx, val = csr_from_coo(m, n, rows, np.concatenate([cols, cols]), np.ones(2 * n))
    return dict(m=m, n=n, m1=m, row_ptr=row_ptr, col_idx=col_idx, val=val,
                c=family["cost"].reshape(-1).copy(), q=np.concatenate([s, d]), l=np.zeros(n),
                u=np.full(n, np.inf), features=np.concatenate([s, d]))


def pagerank(n, seed=0, out_degree=6, damping=0.85, dense_ineq_row=False):
    """A PageRank-shaped LP (the LP form of the PageRank problem, here on a random graph;
    only the shape of the paper's rand_1m / rand_10m instances is reproduced: n columns,
    n + 1 rows, about 8 nonzeros per column).

    Graph: node j links to ``out_degree`` distinct random nodes other than itself, so the
    link matrix S (S_ij = 1 / out_degree for a link j -> i) is column-stochastic.
    LP over x >= 0 with c = 0:
        row 0 (equality):        sum_j x_j = 1          (a dense row)
        rows 1..n (inequality):  x_i - damping (S x)_i >= (1 - damping) / n
    Summing the inequality rows gives (1 - damping) sum x >= 1 - damping, an equality
    once sum x = 1, so every row is tight and the only feasible point is the PageRank
    vector x* = (1 - damping)/n (I - damping S)^-1 1 (returned as x_star; obj_star = 0).
    dense_ineq_row adds the redundant inequality sum_j x_j >= 1/2 (a second dense row,
    in the inequality block)."""
    import scipy.sparse as sps
    import scipy.sparse.linalg as spla
    rng = np.random.default_rng(seed)
    d = int(out_degree)
    src = np.repeat(np.arange(n), d)
    # d distinct targets per node, none equal to the node: uniform draws from the other
    # n - 1 nodes, rows with a repeated target drawn again
    t = rng.integers(0, n - 1, size=(n, d))
    while True:
        ts = np.sort(t, axis=1)
        bad = np.nonzero((ts[:, 1:] == ts[:, :-1]).any(axis=1))[0]
        if bad.size == 0:
            break
        t[bad] = rng.integers(0, n - 1, size=(bad.size, d))
    t = t + (t >= np.arange(n)[:, None])
    dst = t.reshape(-1)
    S = sps.csr_matrix((np.full(n * d, 1.0 / d), (dst, src)), shape=(n, n))
    Gm = (sps.identity(n, format="csr") - damping * S).tocsr()
    rows = [sps.csr_matrix(np.ones((1, n)))]
    m1 = 1
    q = [1.0]
    rows.append(Gm)
    q.extend([(1.0 - damping) / n] * n)
    if dense_ineq_row:
        rows.append(sps.csr_matrix(np.ones((1, n))))
        q.append(0.5)
    K = sps.vstack(rows, format="csr")
    K.sort_indices()
    if n <= 20000:
        x_star = spla.spsolve(Gm.tocsc(), np.full(n, (1.0 - damping) / n))
    else:   # power iteration: the error shrinks by the damping factor per step
        x_star = np.full(n, 1.0 / n)
        for _ in range(250):
            x_star = damping * (S @ x_star) + (1.0 - damping) / n
    m = K.shape[0]
    return dict(m=m, n=n, m1=m1, row_ptr=K.indptr.astype(np.int64), col_idx=K.indices.astype(np.int32),
                val=K.data.astype(np.float64), c=np.zeros(n), q=np.asarray(q, dtype=np.float64),
                l=np.zeros(n), u=np.full(n, np.inf), x_star=x_star, obj_star=0.0)
