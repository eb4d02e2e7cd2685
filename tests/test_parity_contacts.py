"""The contact-record comparison of the parity tests (host logic, no GPU): records are
matched by geom pair and position whatever their order, and a mistake planted in one
side's records (swapped forces, a moved point, a contact on another pair) is caught."""
import numpy as np

from parity import contact_errors, match_contacts


def _records(rng, n, pairs):
    r = np.zeros((n, 24))
    r[:, 0:2] = pairs
    r[:, 4] = -rng.uniform(1e-4, 5e-4, n)
    r[:, 5:8] = rng.uniform(-1, 1, (n, 3))
    r[:, 8:11] = [0.0, 0.0, 1.0]
    r[:, 21:24] = rng.normal(0, 50.0, (n, 3))
    return r


def test_matching_ignores_record_order():
    rng = np.random.default_rng(0)
    a = _records(rng, 6, [[0, 3]] * 4 + [[0, 5]] * 2)
    perm = rng.permutation(6)
    err = contact_errors(a[perm], a, mtot=10.0)
    assert err == {"cpos": 0.0, "cnormal": 0.0, "cdist": 0.0, "cforce": 0.0}
    pairs = match_contacts(a[perm], a)
    assert sorted(perm[i] == j for i, j in pairs) == [True] * 6


def test_swapped_forces_within_a_pair_are_caught():
    rng = np.random.default_rng(1)
    a = _records(rng, 4, [[0, 3]] * 4)
    b = a.copy()
    b[[0, 1], 21:24] = b[[1, 0], 21:24]          # same total force, different split
    assert np.allclose(a[:, 21:24].sum(0), b[:, 21:24].sum(0))
    err = contact_errors(b, a, mtot=1.0)
    assert err["cforce"] > 1e-2 and err["cpos"] == 0.0


def test_moved_point_and_changed_penetration_are_measured():
    rng = np.random.default_rng(2)
    a = _records(rng, 3, [[0, 3]] * 3)
    b = a.copy()
    b[2, 5] += 2e-3                               # 2 mm along x
    b[1, 4] -= 3e-5                               # 30 um deeper
    err = contact_errors(b, a, mtot=1.0)
    assert abs(err["cpos"] - 2e-3 / max(1.0, np.abs(a[2, 5:8]).max())) < 1e-12
    assert abs(err["cdist"] - 3e-5 / 0.1) < 1e-12


def test_same_count_on_other_pairs_is_a_mismatch():
    rng = np.random.default_rng(3)
    a = _records(rng, 3, [[0, 3], [0, 3], [0, 5]])
    b = a.copy()
    b[2, 1] = 3                                   # third contact reported on pair (0, 3)
    assert contact_errors(b, a, mtot=1.0) is None
    assert contact_errors(a[:2], a, mtot=1.0) is None
