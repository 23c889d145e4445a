"""The 2D kernels split a linear cell index c = cy nx + cx by a multiply and shifts
instead of a division: Granlund and Montgomery's method for an invariant divisor
(PLDI 1994, Fig. 4.1).  Written out here in exact integers, as the host (multiplier,
shift) and the device (quotient) compute it, and checked against floor division for
every grid width the 2D path accepts in shape and for indices at and around every
multiple of the width up to the largest grid (nx (ny + 1) <= 2^30)."""
import numpy as np

M32 = (1 << 32) - 1


def make_div(nx):
    l = 0
    while (1 << l) < nx:
        l += 1
    m = ((1 << 32) * ((1 << l) - nx)) // nx + 1
    assert 0 <= m <= M32
    return m, l - 1


def div(n, m, s):
    t = (m * n) >> 32  # mulhi of two 32-bit words
    return ((t + (((n - t) & M32) >> 1)) & M32) >> s


def test_quotients_match_floor_division():
    rng = np.random.default_rng(1994)
    widths = list(range(2, 2050)) + [1 << k for k in range(1, 31)] + \
        [int(x) for x in rng.integers(2, 1 << 30, 200)] + [3 * 5 * 7 * 11 * 13, 65535, 65537]
    for nx in widths:
        m, s = make_div(nx)
        top = 1 << 30
        ks = np.unique(np.concatenate([np.arange(0, 40), rng.integers(0, top // nx + 1, 40),
                                       [top // nx, top // nx + 1]]))
        ns = {0, 1, top - 1, top, M32 >> 1}
        for k in ks:
            for d in (-1, 0, 1, nx - 1):
                v = int(k) * nx + d
                if 0 <= v <= M32 >> 1:
                    ns.add(v)
        ns.update(int(x) for x in rng.integers(0, 1 << 31, 64))
        for n in ns:
            assert div(n, m, s) == n // nx, (nx, n)
