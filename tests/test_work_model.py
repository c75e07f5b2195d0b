"""The roofline's work model (paper_2211_12265_gb300/work.py) against the
oracle's own counters on the same seeded tasks: permutations, butterflies,
pointwise products and coefficients of Alg 2 and Alg 3."""
import numpy as np
import pytest

from paper_2211_12265_gb300 import work as WK
from paper_2211_12265_gb300 import workload as W


@pytest.mark.parametrize("level", [2, 3, 5])
def test_sign_and_verify_counts(orc, level):
    n = 24
    seeds = W.seeds(n, 40 + level)
    lens = W.message_lengths(n, 40 + level, "uniform", 0, 600)
    msg, off = W.messages(lens, 40 + level)
    pk, sk = orc.keygen_batch(level, seeds)
    orc.counters_reset()
    sig, st, it = orc.sign_batch(level, sk, msg, off)
    c = orc.counters()
    w = WK.sign_work(level, it, lens)
    # exact where the algorithm is data-independent
    assert w["coefficients"] == c["coefficients"]
    # permutations: SampleInBall / ExpandA may rarely squeeze one more block
    assert w["permutations"] <= c["permutations"] <= w["permutations"] * 1.01
    # the masking term (Alg 2) is counted once per task by the model,
    # for every iteration that passes the first checks by the oracle
    assert w["butterflies"] <= c["butterflies"] <= w["butterflies"] * 1.10
    assert w["pointwise"] <= c["pointwise"] <= w["pointwise"] * 1.10
    orc.counters_reset()
    ok = orc.verify_batch(level, pk, msg, off, sig)
    c = orc.counters()
    assert ok.all()
    v = WK.verify_work(level, lens)
    assert v["coefficients"] == c["coefficients"]
    assert v["butterflies"] == c["butterflies"] and v["pointwise"] == c["pointwise"]
    assert v["permutations"] <= c["permutations"] <= v["permutations"] * 1.01


def test_int_ops_weights():
    w = dict(permutations=1, butterflies=0, pointwise=0, coefficients=0)
    assert WK.int_ops(w) == 24 * 190
