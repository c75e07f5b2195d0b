"""Hardware probes of the integer roofline: issue rates of the instruction
classes the kernels use and the throughput of the four Keccak-f[1600] forms.

Usage: ``python -m paper_2211_12265_gb300.probe`` prints one JSON object.
"""
from __future__ import annotations

import json


def measure(device: int = 0) -> dict:
    from . import dil
    with dil.Context(device) as ctx:
        issue = {name: dil.dil_test_issue_rate(ctx.handle, op) for name, op in dil.ISSUE_OPS.items()}
        forms = {name: dil.dil_test_keccak_rate(ctx.handle, form)
                 for name, form in (("one_state_25_lanes", 1), ("two_states_interleaved", 2),
                                    ("six_states_row_layout", 6), ("sixteen_states_two_threads", 16))}
    return {"issue_thread_ops_per_sm_clk": issue, "keccak_sm_clk_per_state_round": forms}


if __name__ == "__main__":
    print(json.dumps(measure()))
