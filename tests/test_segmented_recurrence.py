"""The direct 2D solver's Thomas substitutions run in segments side by side: each
first-order recurrence x_j = m_j (x_{j-1} + v_j) (forward) and u_j = v_j + m_j u_{j+1}
(back) is solved in every segment from a zero start, the value entering each segment
follows from the segments' ends, and x = x~ + P x_in with P the product of the segment's
multipliers up to (forward) or from (back) the row.  Written out here in FP64 as the
kernel and its host tables do it, and held to the sequential Thomas solve of the
periodic-x / Dirichlet-y mode systems (4 - 2 cos(2 pi k / nx)) u_j - u_{j-1} - u_{j+1} =
b_j, for row counts that leave short, single-row and empty segments, and to
numpy's dense solve."""
import numpy as np
import pytest

SEGS = 32


def multipliers(a, ny):
    m = np.zeros(ny + 1)
    prev = 0.0
    for j in range(1, ny):
        prev = 1.0 / (a - prev)
        m[j] = prev
    return m


def thomas(m, b, ny):
    d = np.zeros(ny + 1)
    x = 0.0
    for j in range(1, ny):
        x = (b[j] + x) * m[j]
        d[j] = x
    u = np.zeros(ny + 1)
    x = 0.0
    for j in range(ny - 1, 0, -1):
        x = x * m[j] + d[j]
        u[j] = x
    return u


def segmented(m, b, ny):
    L = (ny - 1 + SEGS - 1) // SEGS
    seg_f, seg_b = np.zeros(ny + 1), np.zeros(ny + 1)
    for j0 in range(1, ny, L):  # the host tables
        j1 = min(ny, j0 + L)
        f = g = 1.0
        for j in range(j0, j1):
            f *= m[j]
            seg_f[j] = f
        for j in range(j1 - 1, j0 - 1, -1):
            g *= m[j]
            seg_b[j] = g
    spec = np.array(b, dtype=np.float64)
    ends = np.zeros(SEGS)
    for t in range(SEGS):  # 1. forward from zero
        x = 0.0
        for j in range(1 + t * L, min(ny, 1 + (t + 1) * L)):
            x = (spec[j] + x) * m[j]
            spec[j] = x
        ends[t] = x
    inn = np.zeros(SEGS)  # 2. the value entering each segment
    c = 0.0
    for t in range(SEGS):
        inn[t] = c
        e = min(ny, 1 + (t + 1) * L) - 1
        if 1 + t * L <= e:
            c = ends[t] + seg_f[e] * c
    for t in range(SEGS):  # 3. forward completed, back from zero, top down
        u = 0.0
        for j in range(min(ny, 1 + (t + 1) * L) - 1, 1 + t * L - 1, -1):
            dj = spec[j] + seg_f[j] * inn[t]
            u = u * m[j] + dj
            spec[j] = u
        ends[t] = u
    c = 0.0  # 4. the back value entering each segment from above
    for t in range(SEGS - 1, -1, -1):
        inn[t] = c
        b0 = 1 + t * L
        if b0 <= min(ny, b0 + L) - 1:
            c = ends[t] + seg_b[b0] * c
    for t in range(SEGS):  # 5. back completed
        for j in range(1 + t * L, min(ny, 1 + (t + 1) * L)):
            spec[j] += seg_b[j] * inn[t]
    return spec


@pytest.mark.parametrize("ny", [2, 3, 9, 33, 48, 64, 100, 1025])
@pytest.mark.parametrize("k_over_nx", [0.0, 1.0 / 64, 0.25, 0.5])
def test_segmented_substitutions_match_thomas(ny, k_over_nx):
    rng = np.random.default_rng(ny)
    a = 4.0 - 2.0 * np.cos(2.0 * np.pi * k_over_nx)
    m = multipliers(a, ny)
    b = np.zeros(ny + 1)
    b[1:ny] = rng.standard_normal(ny - 1)
    ref = thomas(m, b, ny)
    got = segmented(m, b, ny)
    scale = np.abs(ref).max()
    assert np.abs(got[1:ny] - ref[1:ny]).max() <= 1e-13 * scale
    # and the system itself: the Thomas solve is right
    n = ny - 1
    A = np.diag(np.full(n, a)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)
    dense = np.linalg.solve(A, b[1:ny])
    assert np.abs(ref[1:ny] - dense).max() <= 1e-10 * max(1.0, np.abs(dense).max())
