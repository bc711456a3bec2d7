"""The CPU oracle against what the paper and the mathematics fix (no GPU)."""
import types

import pytest

import pins


@pytest.fixture(scope="module")
def ns(oracle_ns):
    return types.SimpleNamespace(Oracle=oracle_ns.Oracle, thomas=oracle_ns.thomas,
                                 column_solve=oracle_ns.column_solve, column_solve2=oracle_ns.column_solve2,
                                 bf16=oracle_ns.bf16)


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(ns, pin):
    pin(ns)
