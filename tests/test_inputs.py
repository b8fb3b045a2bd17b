"""Seeded input generators: splitmix64 / xoshiro256** from their published
definitions (first splitmix64 outputs for seed 0 are the published values; the
first xoshiro256** outputs from a set state are worked by hand from the
recurrence)."""
import synthetic as inputs


def test_splitmix64_seed_zero_published_sequence():
    g = inputs.Xoshiro256ss(0)
    assert g.s[:3] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_forest_parameters_in_ranges():
    trees = inputs.forest_trees(64)
    assert len(trees) == 64
    for t in trees:
        assert 4 <= t["Jmax"] <= 8 and t["Jmin"] == 2
        assert 1e-5 <= t["eps"] <= 1e-3
        assert 0.02 <= t["ic_params"][3] <= 0.1
        assert all(-1 <= u <= 1 for u in t["rhs_params"][:2])
    assert inputs.forest_trees(4, seed=5) == inputs.forest_trees(4, seed=5)


def test_xoshiro256ss_step_from_a_set_state():
    # from the state (1, 2, 3, 4): the first output is rotl(2 * 5, 7) * 9 = 11520,
    # the second 0 (s[1] becomes 2 ^ 2), the third rotl(262149 * 5, 7) * 9 =
    # 1509978240, worked by hand from the published recurrence
    g = inputs.Xoshiro256ss(0)
    g.s = [1, 2, 3, 4]
    assert [g.next() for _ in range(3)] == [11520, 0, 1509978240]
    u = [inputs.Xoshiro256ss(7).uniform() for _ in range(2)]
    assert u[0] == u[1] and 0.0 <= u[0] < 1.0
