"""The oracle pinned against closed forms, LAPACK special cases and method invariants.

Planted-mistake builds (``-DORC_MUTANT=k``) show each pin set is sensitive: every
mutant must fail at least one pin.
"""
import numpy as np
import pytest

import pins
from oracle import Oracle


@pytest.mark.parametrize("pin", pins.ALL_PINS + [pins.pin_generator_2x2], ids=lambda f: f.__name__)
def test_pin(orc, pin):
    ok, detail = pin(orc)
    assert ok, detail


MUTANTS = {
    1: "beta dropped from the direction update",
    2: "sign of the W mu term flipped",
    3: "bhat formed with AW instead of W",
    4: "Jacobi preconditioner multiplies by diag(A) instead of its inverse",
    5: "POD lift without 1/sigma",
    6: "energy criterion on sigma instead of sigma^2",
    7: "Cholesky reads a wrong, scaled entry",
    8: "residual update with p instead of A p",
    9: "wrong sign in the eigenvector rotation",
    10: "SpMV drops the first entry of each row",
}


@pytest.mark.parametrize("k", sorted(MUTANTS))
def test_planted_mistake_is_caught(k, tmp_path):
    mut = Oracle(mutant=k, out_dir=str(tmp_path))
    failed = []
    for pin in pins.ALL_PINS:
        try:
            ok, detail = pin(mut)
        except Exception as e:  # a crash or a numpy error also counts as caught
            ok, detail = False, repr(e)
        if not ok:
            failed.append(pin.__name__)
    assert failed, f"mutant {k} ({MUTANTS[k]}) passed every pin"
