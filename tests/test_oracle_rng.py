"""Oracle pins: the counter-based Philox4x32-10 generator and its uniforms."""
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    with open(GOLD) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert orc.philox4x32_10(ctr, key) == out


def test_uniforms_open_interval_and_moments(orc):
    us = np.array([orc.draw_uniforms(7, 3, s, s % 4, 0, 0, orc.KIND_HB, 11) for s in range(4000)]).ravel()
    assert us.min() > 0.0 and us.max() < 1.0
    n = us.size
    assert abs(us.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(us.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / n)


def test_counter_fields_are_independent_streams(orc):
    base = dict(seed=5, lattice_id=2, site=17, mu=1, subgroup=2, attempt=0, kind=orc.KIND_HB, sweep=9)
    ref = orc.draw_uniforms(*base.values())
    for field, alt in [("seed", 6), ("lattice_id", 3), ("site", 18), ("mu", 2), ("subgroup", 1),
                       ("attempt", 1), ("kind", orc.KIND_MOM), ("sweep", 10), ("sweep", 9 + (1 << 32))]:
        d = dict(base)
        d[field] = alt
        assert not np.array_equal(orc.draw_uniforms(*d.values()), ref), field


def test_uniform_is_exact_affine_map_of_the_word(orc):
    # u = (w + 0.5) 2^-32 must be recoverable exactly as an integer word
    ctr = [17, 1 | (2 << 2) | (0 << 4) | (orc.KIND_HB << 12), 9, 0]
    key = [5, 0 ^ 2]
    w = orc.philox4x32_10(ctr, key)
    u = orc.draw_uniforms(5, 2, 17, 1, 2, 0, orc.KIND_HB, 9)
    assert [int(x * 2.0**32 - 0.5) for x in u] == w
