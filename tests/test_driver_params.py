"""The driver's parameter keywords carry the paper's defaults (Sec. 4: one random
vector, 1000 moments, energy scale 10, no VAC or MSD rows), and a run that asks
for VAC or MSD rows without time steps is refused before any GPU work."""
import pytest

pytest.importorskip("torch")
from paper_1705_01387_gb300 import driver  # noqa: E402


def test_defaults():
    p = driver.Params()
    assert (p.calculate_vac, p.calculate_msd) == (False, False)
    assert (p.number_of_random_vectors, p.number_of_moments, p.energy_max) == (1, 1000, 10.0)


def test_time_steps_required():
    with pytest.raises(ValueError):
        driver.run(None, [0.0], driver.Params(calculate_vac=True))
    with pytest.raises(ValueError):
        driver.run(None, [0.0], driver.Params(calculate_msd=True))
