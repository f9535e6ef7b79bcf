"""Seeded synthetic F4-shaped matrices over GF(p).

This module only draws random matrices; it holds none of the reduction's
arithmetic.  Both the CUDA path's tests/benchmarks and the CPU oracle's tests
read their inputs from here.

The shapes follow the statistics the GBLA paper gives for matrices out of F4
and F5 symbolic preprocessing (Sec. 3.1, Sec. 4.2 and Tables 4 and 5): rows are
polynomials, columns monomials in decreasing order; a row's leftmost nonzero
is its pivoting candidate; many rows share a leading column; nonzeros come in
horizontal runs of consecutive columns, and neighbouring rows repeat one
another's pattern (the "vertical pattern").  The paper's own matrices are not
reproduced: only their shape statistics are.

Recipe (all draws from ``numpy.random.Generator(PCG64(seed))``):

1. ``npiv`` distinct leading columns are drawn uniformly in ``[0, n)``.  Each
   designated pivot row has value 1 at its lead.
2. Every row gets ``k = round(density * n * U[1-spread, 1+spread])`` nonzeros
   (clipped to the columns right of its lead) laid out in runs whose lengths
   are uniform in ``run_len``; the runs are spread uniformly over the columns
   right of the lead.
3. With ``group=(gmin, gmax)``, consecutive designated leads form groups whose
   members copy the group's run pattern shifted by the difference of leads
   (a monomial shift), with a fraction ``1 - share`` of runs redrawn.
4. A non-pivot row leads, with probability ``lead_from_pivot``, at the lead of
   a random designated pivot row (an S-pair-like reducible row, copying that
   row's group pattern when groups are on) and otherwise at a random other
   column; its leading value is uniform in ``[1, p-1]``.
5. All other values are uniform in ``[1, p-1]``; rows are shuffled.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class FLSpec:
    m: int
    n: int
    npiv: int
    p: int = 65521
    density: float = 0.04
    run_len: tuple = (4, 32)
    spread: float = 0.5
    lead_from_pivot: float = 0.9
    group: tuple | None = None
    share: float = 0.8
    seed: int = 20160219
    # banded layout (see banded_matrix): band and block widths in pivot
    # columns, fraction of A entries crossing into the next block
    band: int | None = None
    block: int = 4096
    cross: float = 0.05


def _runs(rng, lead, k, n, run_len):
    """Column indices of runs totalling k[i] entries right of lead[i].

    Returns (row_of_entry, col_of_entry) sorted by row then column.
    """
    k = k.astype(np.int64)
    total = int(k.sum())
    if total == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    K = np.cumsum(k)
    mean = 0.5 * (run_len[0] + run_len[1])
    lens = rng.integers(run_len[0], run_len[1] + 1, size=int(total / mean * 1.25) + 16)
    C = np.cumsum(lens)
    while C[-1] < total:
        more = rng.integers(run_len[0], run_len[1] + 1, size=len(lens))
        lens = np.concatenate([lens, more])
        C = np.cumsum(lens)
    # Piece boundaries: run boundaries of one global stream cut at row ends.
    bounds = _sorted_unique(np.concatenate([C[C < total], K[:-1]]))
    bounds = bounds[(bounds > 0) & (bounds < total)]
    bounds = np.concatenate([[0], bounds, [total]]).astype(np.int64)
    pstart = bounds[:-1]
    plen = np.diff(bounds)
    prow = np.searchsorted(K, pstart, side="right")
    row_first_slot = K - k
    span = n - lead - 1
    free = span - k
    o = (rng.random(len(pstart)) * (free[prow] + 1)).astype(np.int64)
    o = np.minimum(o, free[prow])
    order = np.lexsort((o, prow))
    o = o[order]
    start_col = lead[prow] + 1 + o + (pstart - row_first_slot[prow])
    within = np.arange(total, dtype=np.int64) - np.repeat(pstart, plen)
    cols = np.repeat(start_col, plen) + within
    rows = np.repeat(prow, plen)
    return rows, cols


def _sorted_unique(a):
    a = np.sort(a, kind="stable")
    if len(a) == 0:
        return a
    keep = np.empty(len(a), bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def _row_counts(rng, nrows, density, n, spread):
    base = density * n
    f = 1.0 + spread * (2.0 * rng.random(nrows) - 1.0)
    return np.maximum(1, np.rint(base * f)).astype(np.int64)


def fl_matrix(spec: FLSpec):
    """Draw one matrix.  Returns (row_ptr int64[m+1], col int32[nnz], val uint16[nnz])."""
    if spec.band is not None:
        return banded_matrix(spec)
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    m, n, npiv, p = spec.m, spec.n, spec.npiv, spec.p
    if not (0 <= npiv <= min(m, n)):
        raise ValueError("need 0 <= npiv <= min(m, n)")
    piv_leads = np.sort(rng.choice(n, size=npiv, replace=False)).astype(np.int64)
    mnp = m - npiv
    # Leads of the non-pivot rows.
    from_piv = rng.random(mnp) < spec.lead_from_pivot if npiv > 0 else np.zeros(mnp, bool)
    which = rng.integers(0, max(npiv, 1), size=mnp)
    lead_np = np.where(from_piv, piv_leads[np.minimum(which, max(npiv - 1, 0))] if npiv else 0,
                       rng.integers(0, n, size=mnp))
    lead = np.concatenate([piv_leads, lead_np]).astype(np.int64)
    k = _row_counts(rng, m, spec.density, n, spec.spread) - 1
    k = np.minimum(k, n - lead - 1)

    if spec.group is None:
        rows, cols = _runs(rng, lead, k, n, spec.run_len)
    else:
        rows, cols = _grouped(rng, spec, lead, k, piv_leads, from_piv, which)

    # Assemble: lead entry first, then the run entries (already sorted).
    counts = np.bincount(rows, minlength=m).astype(np.int64) + 1
    row_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, np.int64)
    col[row_ptr[:-1]] = lead
    # run entries go after the lead of their row
    rank_in_row = np.arange(len(rows), dtype=np.int64) - np.repeat(
        np.concatenate([[0], np.cumsum(counts - 1)[:-1]]), counts - 1)
    col[row_ptr[rows] + 1 + rank_in_row] = cols
    val = rng.integers(1, p, size=nnz).astype(np.int64)
    val[row_ptr[:npiv]] = 1                       # designated pivot rows are monic
    # Shuffle rows.
    perm = rng.permutation(m)
    cnt = counts[perm]
    new_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(cnt, out=new_ptr[1:])
    src = np.repeat(row_ptr[perm], cnt) + (np.arange(nnz, dtype=np.int64) - np.repeat(new_ptr[:-1], cnt))
    return new_ptr, col[src].astype(np.int32), val[src].astype(np.uint16)


def _grouped(rng, spec, lead, k, piv_leads, from_piv, which):
    """Run patterns shared inside groups of consecutive designated leads."""
    n = spec.n
    npiv = len(piv_leads)
    m = len(lead)
    gmin, gmax = spec.group
    # Group ids over designated pivots (consecutive leads).
    sizes = []
    tot = 0
    while tot < npiv:
        s = int(rng.integers(gmin, gmax + 1))
        sizes.append(s)
        tot += s
    gid_piv = np.repeat(np.arange(len(sizes)), sizes)[:npiv]
    gfirst = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    ngroups = len(sizes)
    # Non-pivot rows copying a pivot's pattern join its group; others get own patterns.
    gid_np = np.where(from_piv, gid_piv[np.minimum(which, max(npiv - 1, 0))] if npiv else -1, -1)
    gid = np.concatenate([gid_piv, gid_np]).astype(np.int64)
    # Base pattern per group: drawn right of the group's first lead.
    base_lead = piv_leads[gfirst] if npiv else np.zeros(0, np.int64)
    base_k = np.minimum(_row_counts(rng, ngroups, spec.density, n, spec.spread) - 1, n - base_lead - 1)
    b_rows, b_cols = _runs(rng, base_lead, base_k, n, spec.run_len)
    b_ptr = np.zeros(ngroups + 1, np.int64)
    np.cumsum(np.bincount(b_rows, minlength=ngroups), out=b_ptr[1:])
    # Members: shifted base entries; keep each with probability `share`
    # (run-granular keep via a per-entry draw on the run id), then top up with
    # fresh runs to the member's own count.
    member = np.nonzero(gid >= 0)[0]
    g = gid[member]
    shift = lead[member] - base_lead[g]
    cnt = b_ptr[g + 1] - b_ptr[g]
    e_row = np.repeat(member, cnt)
    e_src = np.repeat(b_ptr[g], cnt) + (np.arange(int(cnt.sum()), dtype=np.int64) - np.repeat(
        np.concatenate([[0], np.cumsum(cnt)[:-1]]), cnt))
    e_col = b_cols[e_src] + np.repeat(shift, cnt)
    # run id of each base entry: a new run starts where columns are not consecutive
    brk = np.ones(len(b_cols), bool)
    brk[1:] = (b_cols[1:] != b_cols[:-1] + 1) | (b_rows[1:] != b_rows[:-1])
    run_id = np.cumsum(brk) - 1
    keep_run = rng.random(int(run_id[-1]) + 1 if len(run_id) else 0) < spec.share
    keep = (e_col > np.repeat(lead[member], cnt)) & (e_col < n) & keep_run[run_id[e_src]] if len(e_src) else np.zeros(0, bool)
    e_row, e_col = e_row[keep], e_col[keep]
    have = np.bincount(e_row, minlength=m)
    # Fresh runs: rows outside groups get their whole count; members top up.
    need = np.maximum(k - have, 0)
    f_rows, f_cols = _runs(rng, lead, need, n, spec.run_len)
    rows = np.concatenate([e_row, f_rows])
    cols = np.concatenate([e_col, f_cols])
    # Deduplicate and sort per row.
    key = _sorted_unique(rows * (n + 1) + cols)
    rows = key // (n + 1)
    cols = key % (n + 1)
    return rows.astype(np.int64), cols.astype(np.int64)


def _assemble(rng, m, p, lead, rows, cols, monic_rows):
    """CSR of rows with leading column lead[i] and other entries (rows, cols)
    (sorted by row then column, all right of the lead); values uniform in
    [1, p-1], the leads of monic_rows set to 1; rows shuffled."""
    counts = np.bincount(rows, minlength=m).astype(np.int64) + 1
    row_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, np.int64)
    col[row_ptr[:-1]] = lead
    rank_in_row = np.arange(len(rows), dtype=np.int64) - np.repeat(
        np.concatenate([[0], np.cumsum(counts - 1)[:-1]]), counts - 1)
    col[row_ptr[rows] + 1 + rank_in_row] = cols
    del rank_in_row
    val = rng.integers(1, p, size=nnz, dtype=np.int64).astype(np.uint16)
    val[row_ptr[monic_rows]] = 1
    perm = rng.permutation(m)
    cnt = counts[perm]
    new_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(cnt, out=new_ptr[1:])
    src = np.repeat(row_ptr[perm] - new_ptr[:-1], cnt) + np.arange(nnz, dtype=np.int64)
    return new_ptr, col[src].astype(np.int32), val[src]


def banded_matrix(spec: FLSpec):
    """A matrix whose A block is banded and nearly block-diagonal, with rows
    in multiline pairs (the large F4 shape of Sec. 4.2).

    Recipe (``numpy.random.Generator(PCG64(seed))``):

    1. ``npiv`` distinct pivot columns P (sorted) are drawn uniformly in
       [0, n); Q are the other columns.  Pivot row i leads at P[i] with a 1.
    2. Each row gets ``k = density * n * U[1-spread, 1+spread]`` entries
       right of its lead, a share npiv/n of them at pivot columns (the A or C
       part) and the rest at the other columns (B or D), in runs of lengths
       ``run_len``.  A-part runs lie in pivot indices (i, i + band], cut at the
       end of i's block of ``block`` pivot indices; a fraction ``cross`` of
       them lies in the next block.  B-part runs lie in the window of
       ``block * (n - npiv) / npiv`` other columns that follows the lead.
    3. Pivot rows come in pairs (2q, 2q + 1): the second copies the runs of
       the first that lie right of its own lead, each run kept with
       probability ``share``, and is topped up with fresh runs to its count.
    4. The other m - npiv rows lead, with probability ``lead_from_pivot``, at
       the lead of a random pivot row, else at a random other column (their
       lead value uniform in [1, p-1]), and get runs by the same rule from
       their lead.
    5. All other values are uniform in [1, p-1]; rows are shuffled.
    """
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    m, n, npiv, p = spec.m, spec.n, spec.npiv, spec.p
    if not (0 < npiv <= min(m, n)):
        raise ValueError("need 0 < npiv <= min(m, n)")
    band, block = int(spec.band), int(spec.block)
    P = np.sort(rng.choice(n, size=npiv, replace=False)).astype(np.int64)
    is_piv = np.zeros(n, bool)
    is_piv[P] = True
    Q = np.nonzero(~is_piv)[0].astype(np.int64)
    nq = len(Q)
    wb = max(1, int(block * nq / npiv))
    mnp = m - npiv
    from_piv = rng.random(mnp) < spec.lead_from_pivot
    which = rng.integers(0, npiv, size=mnp)
    lead_np = np.where(from_piv, P[which], Q[rng.integers(0, max(nq, 1), size=mnp)] if nq else P[which])
    lead = np.concatenate([P, lead_np]).astype(np.int64)
    # first pivot index and first other-column index right of each lead
    ia = np.searchsorted(P, lead, side="right")
    ib = np.searchsorted(Q, lead, side="right")
    k = _row_counts(rng, m, spec.density, n, spec.spread) - 1
    ka = np.rint(k * (npiv / n)).astype(np.int64)
    kb = k - ka
    kc = np.rint(ka * spec.cross).astype(np.int64)
    ka -= kc
    blk_end = np.minimum((np.maximum(ia - 1, 0) // block + 1) * block, npiv)
    hi_a = np.minimum(ia + band, blk_end)
    ka = np.clip(np.minimum(ka, hi_a - ia), 0, None)
    hi_c = np.minimum(blk_end + block, npiv)
    kc = np.clip(np.minimum(kc, hi_c - blk_end), 0, None)
    hi_b = np.minimum(ib + wb, nq)
    kb = np.clip(np.minimum(kb, hi_b - ib), 0, None)
    # runs inside windows: _runs places k[i] entries in runs right of
    # lead[i] and below its (per-row) bound
    ra, ca = _runs(rng, ia - 1, ka, hi_a, spec.run_len)
    rc, cc = _runs(rng, blk_end - 1, kc, hi_c, spec.run_len)
    rb, cb = _runs(rng, ib - 1, kb, hi_b, spec.run_len)
    rows = np.concatenate([ra, rc, rb])
    cols = np.concatenate([P[ca], P[cc], Q[cb]])
    del ra, ca, rc, cc, rb, cb
    # multiline pairs: row 2q+1 shares the runs of row 2q right of its lead
    key = rows * (n + 1) + cols
    first = rows < npiv
    first &= (rows % 2 == 0) & (rows + 1 < npiv)
    fr, fc = rows[first], cols[first]
    brk = np.ones(len(fc), bool)
    if len(fc):
        brk[1:] = (fc[1:] != fc[:-1] + 1) | (fr[1:] != fr[:-1])
    run_id = np.cumsum(brk) - 1
    keep_run = rng.random(int(run_id[-1]) + 1 if len(run_id) else 0) < spec.share
    keep = keep_run[run_id] & (fc > lead[fr + 1]) if len(fc) else np.zeros(0, bool)
    second_rows = fr[keep] + 1
    second_cols = fc[keep]
    del fr, fc, brk, run_id, keep
    drop = (rows % 2 == 1) & (rows < npiv)
    # the second row's own runs fill up to its count after the shared ones
    have = np.bincount(second_rows, minlength=m)
    own = np.nonzero(drop)[0]
    rank_in_row = np.arange(len(rows), dtype=np.int64) - np.repeat(
        np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=m))[:-1]]), np.bincount(rows, minlength=m))
    keep_own = ~drop | (rank_in_row < np.maximum(np.bincount(rows, minlength=m) - have, 0)[rows])
    del rank_in_row, own
    rows = np.concatenate([rows[keep_own], second_rows])
    cols = np.concatenate([cols[keep_own], second_cols])
    del keep_own, second_rows, second_cols, key
    key = _sorted_unique(rows * (n + 1) + cols)
    rows = key // (n + 1)
    cols = key % (n + 1)
    del key
    return _assemble(rng, m, p, lead, rows, cols, np.arange(npiv))


# Named workloads (sizes from the F4 shape statistics quoted above).
WORKLOADS = {
    # 2,000 x 3,000, 1,200 pivots, 4% density, runs of 4-32: the small case.
    "fl_2000x3000": FLSpec(m=2000, n=3000, npiv=1200, density=0.04, run_len=(4, 32), seed=20160219),
    # 40,000 x 60,000, 30,000 pivots, 1.5% density, 2-8 runs per row,
    # groups of 2-16 rows sharing ~80% of their pattern.
    "fl_40000x60000": FLSpec(m=40000, n=60000, npiv=30000, density=0.015, run_len=(112, 450),
                             group=(2, 16), share=0.8, seed=20160220),
    # 150,000 x 200,000, 120,000 pivots, 0.5% density (~150M nonzeros), rows
    # in multiline pairs sharing ~90% of their pattern, A banded (2,048
    # pivot columns) in diagonal blocks of 4,096 with 5% cross-block entries.
    "fl_150000x200000": FLSpec(m=150000, n=200000, npiv=120000, density=0.005, run_len=(4, 32),
                               share=0.9, band=2048, block=4096, cross=0.05, seed=20160221),
    # 40,000 x 120,000, 15,000 pivots, 0.02% density (24 entries per row in
    # runs of 1-3): few pivots and short rows, so that the Schur complement
    # stays sparse (about 4% of its entries nonzero) -- the case the sparse
    # SGE of the echelon step is for.
    "fl_sparse_d_40000x120000": FLSpec(m=40000, n=120000, npiv=15000, density=0.0002, run_len=(1, 3),
                                       seed=1602),
}


def mixed_batch(count: int, seed: int, rows=(500, 20000), primes=(65521, 32003)):
    """Specs of a batch of F4-shaped matrices of uneven sizes: rows
    log-uniform in ``rows``, columns 1.3-1.6 x rows, 60-80% designated pivots,
    density 1-5%, runs of 4-32, p drawn from ``primes``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        m = int(np.exp(rng.uniform(np.log(rows[0]), np.log(rows[1]))))
        ncols = int(m * rng.uniform(1.3, 1.6))
        npiv = int(m * rng.uniform(0.6, 0.8))
        out.append(FLSpec(m=m, n=ncols, npiv=npiv, p=int(rng.choice(list(primes))),
                          density=float(rng.uniform(0.01, 0.05)), run_len=(4, 32), seed=seed * 1000 + i))
    return out


def workload(name: str, **overrides):
    spec = WORKLOADS[name]
    if overrides:
        spec = dataclasses.replace(spec, **overrides)
    return spec


def scaled(name: str, scale: float, seed: int | None = None) -> FLSpec:
    """The named workload with rows, columns and pivots scaled by ``scale``."""
    s = WORKLOADS[name]
    m = max(2, int(round(s.m * scale)))
    n = max(2, int(round(s.n * scale)))
    npiv = max(1, min(m, n, int(round(s.npiv * scale))))
    rl = (max(1, int(round(s.run_len[0] * min(1.0, scale * 4)))), max(1, int(round(s.run_len[1] * min(1.0, scale * 4)))))
    return dataclasses.replace(s, m=m, n=n, npiv=npiv, run_len=(min(rl), max(rl)),
                               seed=s.seed if seed is None else seed)


def random_csr(rng, m, n, p, density):
    """Unstructured random sparse matrix (for edge-case tests)."""
    mask = rng.random((m, n)) < density
    vals = rng.integers(1, p, size=(m, n))
    dense = np.where(mask, vals, 0)
    return dense_to_csr(dense)


def dense_to_csr(dense):
    dense = np.asarray(dense)
    m, n = dense.shape
    nzr, nzc = np.nonzero(dense)
    row_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(np.bincount(nzr, minlength=m), out=row_ptr[1:])
    return row_ptr, nzc.astype(np.int32), dense[nzr, nzc].astype(np.uint16)


def csr_to_dense(m, n, row_ptr, col, val):
    out = np.zeros((m, n), np.int64)
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    out[rows, np.asarray(col, np.int64)] = np.asarray(val, np.int64)
    return out


# ------------------------------------------------------------- matrix files
# Writers of the paper's two binary matrix files (Sec. 3.2, Table 2), used to
# feed matrices to the file readers in tests: little-endian, fields in the
# table's order.

def encode_format1(m, n, p, row_ptr, col, val) -> bytes:
    """Format 1: u32 m, n, p; u64 nnz; u16 data; u32 cols; u32 row lengths."""
    row_ptr = np.asarray(row_ptr, np.int64)
    nnz = int(row_ptr[-1])
    parts = [np.array([m, n, p], "<u4").tobytes(), np.array([nnz], "<u8").tobytes(),
             np.asarray(val, "<u2").tobytes(), np.asarray(col, "<u4").tobytes(),
             np.diff(row_ptr).astype("<u4").tobytes()]
    return b"".join(parts)


_CODES = {"u1": (1, 0), "u2": (1, 1), "u4": (1, 2), "u8": (1, 3),
          "i1": (0, 0), "i2": (0, 1), "i4": (0, 2), "i8": (0, 3)}


def encode_format2(m, n, p, row_ptr, col, val, vtype=None) -> bytes:
    """Format 2.  Rows whose coefficient sequences are equal share one
    polynomial (numbered in order of first use); each row's columns are cut
    into maximal runs of consecutive columns, a run of s >= 2 written as the
    pair (first, s), a lone column c as c | 2^31.  ``vtype`` is a numpy type
    code (default: the smallest unsigned type that holds p - 1); a signed type
    stores the residues balanced, in (-p/2, p/2]."""
    row_ptr = np.asarray(row_ptr, np.int64)
    col = np.asarray(col, np.int64)
    val = np.asarray(val, np.int64)
    nnz = int(row_ptr[-1])
    lengths = np.diff(row_ptr)
    if vtype is None:
        vtype = next(t for t, bits in (("u1", 8), ("u2", 16), ("u4", 32), ("u8", 64)) if p - 1 < 1 << bits)
    u, v = _CODES[vtype]
    b = u | (v << 1)
    # polynomials
    poly_of = {}
    polmap = np.zeros(m, np.int64)
    pdata, prow = [], []
    for i in range(m):
        key = val[row_ptr[i]:row_ptr[i + 1]].tobytes()
        j = poly_of.get(key)
        if j is None:
            j = poly_of[key] = len(prow)
            prow.append(int(lengths[i]))
            pdata.append(val[row_ptr[i]:row_ptr[i + 1]])
        polmap[i] = j
    coeffs = np.concatenate(pdata) if pdata else np.zeros(0, np.int64)
    if u == 0:
        coeffs = np.where(coeffs > p // 2, coeffs - p, coeffs)
    # column runs
    rid = np.repeat(np.arange(m), lengths)
    start = np.ones(nnz, bool)
    if nnz:
        start[1:] = (col[1:] != col[:-1] + 1) | (rid[1:] != rid[:-1])
    first = np.nonzero(start)[0]
    size = np.diff(np.append(first, nnz))
    width = np.where(size > 1, 2, 1)
    pos = np.concatenate([[0], np.cumsum(width)[:-1]]) if len(first) else np.zeros(0, np.int64)
    colid = np.zeros(int(width.sum()), np.uint64)
    single = size == 1
    colid[pos[single]] = col[first[single]].astype(np.uint64) | np.uint64(1 << 31)
    colid[pos[~single]] = col[first[~single]].astype(np.uint64)
    colid[pos[~single] + 1] = size[~single].astype(np.uint64)
    parts = [np.array([b, m, n], "<u4").tobytes(), np.array([p, nnz], "<u8").tobytes(),
             lengths.astype("<u4").tobytes(), polmap.astype("<u4").tobytes(),
             np.array([len(colid)], "<u8").tobytes(), colid.astype("<u8").tobytes(),
             np.array([len(prow)], "<u4").tobytes(), np.array([len(coeffs)], "<u8").tobytes(),
             np.asarray(prow, np.int64).astype("<u4").tobytes(), coeffs.astype("<" + vtype).tobytes()]
    return b"".join(parts)
