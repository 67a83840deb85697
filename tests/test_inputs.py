"""The seeded input generators (no method arithmetic in them)."""
import numpy as np

from paper_1510_07328_gb300 import inputs


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 0: first outputs 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4
    z = inputs.splitmix64(0, 2)
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4


def test_uniform_range_and_counter_offsets():
    u = inputs.uniform(7, 1000)
    assert u.min() >= 0.0 and u.max() < 1.0
    np.testing.assert_array_equal(inputs.uniform(7, 10, offset=5), u[5:15])


def test_workload_shapes_and_ranges():
    p = inputs.riemann_1d()
    assert (p.nx, p.ny) == (400, 4) and p.n[0, 199] == 1.0 and p.n[0, 200] == 0.8
    q = inputs.quadrants(64)
    assert q.n.min() >= 0.7 and q.n.max() <= 1.0 and q.t.min() >= 0.02 and q.t.max() <= 0.1
    t = inputs.smooth_t_field(128)
    assert abs(t.min() - 0.01) < 1e-15 and abs(t.max() - 0.2) < 1e-15
    band = inputs.smooth_t_field(128, rows=slice(10, 20))
    np.testing.assert_array_equal(band, t[10:20])
    specs = inputs.batched_specs()
    assert len(specs) == 256
    assert all(256 <= s.nx <= 8192 and 4 <= s.ny <= 64 for s in specs)
    assert all(1.05 <= s.n_left <= 2.0 and 0.01 <= s.t <= 0.2 and 0.55 <= s.tau <= 1.0 for s in specs)
    n, tt = inputs.surrogate_set(1000)
    assert n.min() >= 0.5 and n.max() <= 2.0 and tt.min() >= 0.005 and tt.max() <= 0.3
