"""Measured parity errors.

Every GPU-versus-oracle comparison goes through ``check``.  It asserts the
bound, and it also records the error that was measured, so that a run states
each result's error against the FP64 oracle next to its bound, not only that
the bound held.  ``tests/conftest.py`` prints the records at the end of the
session.  When ``DNNMG_PARITY_LOG`` names a file, it also writes them there as
JSON lines.
"""

import os

RECORDS = []


def _test_id():
    cur = os.environ.get("PYTEST_CURRENT_TEST", "")
    return cur.rsplit(" (", 1)[0]


def record(quantity, err, bound, prec=None, step=None, **extra):
    rec = {"test": _test_id(), "quantity": quantity, "err": float(err), "bound": float(bound)}
    if prec is not None:
        rec["prec"] = prec
    if step is not None:
        rec["step"] = int(step)
    rec.update(extra)
    RECORDS.append(rec)
    return rec


def check(quantity, err, bound, prec=None, step=None, **extra):
    """Record a measured error and assert that it is within its bound."""
    record(quantity, err, bound, prec=prec, step=step, **extra)
    assert err <= bound, (quantity, prec, step, err, bound)
