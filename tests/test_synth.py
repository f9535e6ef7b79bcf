"""The seeded input generator against the recipe it documents (F4-shaped
matrices: designated pivot rows with distinct leads, reducible rows leading at
a designated lead with probability lead_from_pivot, about density * n entries
per row in runs of consecutive columns, values in [1, p), rows shuffled,
deterministic per seed)."""
import numpy as np
import pytest

from paper_1602_06097_gb300 import synth


def leads_and_lengths(rp, c):
    nz = np.diff(rp) > 0
    return c[rp[:-1][nz]].astype(np.int64), np.diff(rp)


@pytest.mark.parametrize("name,scale", [("fl_2000x3000", 1.0), ("fl_40000x60000", 0.05)])
def test_valid_csr_and_value_range(name, scale):
    spec = synth.workload(name) if scale == 1.0 else synth.scaled(name, scale)
    rp, c, v = synth.fl_matrix(spec)
    assert rp[0] == 0 and len(rp) == spec.m + 1 and np.all(np.diff(rp) >= 1)
    assert len(c) == len(v) == rp[-1]
    for i in range(0, spec.m, max(1, spec.m // 200)):
        row = c[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0) and row[0] >= 0 and row[-1] < spec.n
    assert v.min() >= 1 and int(v.max()) < spec.p


def test_deterministic_per_seed():
    spec = synth.workload("fl_2000x3000")
    a, b = synth.fl_matrix(spec), synth.fl_matrix(spec)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    c = synth.fl_matrix(synth.workload("fl_2000x3000", seed=spec.seed + 1))
    assert not np.array_equal(a[1], c[1])


def test_leads_and_density_follow_the_recipe():
    spec = synth.workload("fl_2000x3000")
    rp, c, v = synth.fl_matrix(spec)
    lead, length = leads_and_lengths(rp, c)
    distinct = len(np.unique(lead))
    mnp = spec.m - spec.npiv
    # npiv designated distinct leads, plus the other rows' leads that are not one of them
    assert spec.npiv <= distinct <= spec.npiv + 2 * (1 - spec.lead_from_pivot) * mnp
    # rows leading at a column some other row also leads at: the designated
    # leads shared by reducible rows
    _, counts = np.unique(lead, return_counts=True)
    shared_rows = int(counts[counts > 1].sum()) - int((counts > 1).sum())
    assert abs(shared_rows / mnp - spec.lead_from_pivot) < 0.08
    mean = length.mean()
    assert 0.5 * spec.density * spec.n <= mean <= 1.5 * spec.density * spec.n


def test_runs_of_consecutive_columns():
    spec = synth.workload("fl_2000x3000")
    rp, c, _ = synth.fl_matrix(spec)
    runs = []
    for i in range(0, spec.m, 10):
        row = c[rp[i] + 1:rp[i + 1]].astype(np.int64)     # the lead stands apart
        if len(row) < 2:
            continue
        cut = np.nonzero(np.diff(row) != 1)[0]
        bounds = np.concatenate([[0], cut + 1, [len(row)]])
        runs.extend(np.diff(bounds))
    runs = np.array(runs)
    lo, hi = spec.run_len
    assert lo <= np.median(runs) <= 2 * hi                  # adjacent runs may merge, ends are clipped
    assert np.mean(runs >= lo) > 0.5
