"""The CPU oracle against its pins (no GPU)."""
import pytest

import pins


@pytest.mark.parametrize("name,fn", pins.ALL_PINS, ids=[n for n, _ in pins.ALL_PINS])
def test_pin(name, fn):
    fn()


def test_worked_example_second_atc_value():
    # Table 2 lists ATC twice (0.62 and 0.77); the example's result must not
    # depend on which value is taken.
    pins.pin_worked_example(atc_value=77)


def test_ed_bfs_three_letters():
    pins.pin_ed_bfs(alphabet=b"ACG", maxlen=4, band_k=(0, 1, 3))


def test_join_recall_reported():
    found, truth = pins.pin_join_precision(seed=32)
    assert found <= truth
