"""The oracle's pins catch plausible mistakes: every mutant of
oracle.mutation_check (a wrong sign, index, factor or a dropped term in a copy
of the oracle's C sources, in the push, gather, ZigZag, fields, filter, wall,
injector and adjoint) makes at least one pin test fail.  The oracle's own
sources are not touched."""
import pytest

from oracle import mutation_check


@pytest.mark.parametrize("name", [m[0] for m in mutation_check.MUTATIONS])
def test_pins_catch_the_planted_mistake(name):
    caught, last = mutation_check.run_one(name)
    assert caught, f"mutant {name} survived the pins: {last}"
