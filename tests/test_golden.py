"""The printed constants of Eq. 1 (tests/golden/paper_constants.json) are the
defaults of the oracle, and, on a GPU, of the library."""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def constants():
    with open(GOLDEN) as f:
        return json.load(f)


def test_oracle_defaults_are_the_printed_constants():
    c = constants()
    assert oracle.PAPER_CONSTANTS == (c["omega_a_per_s"], c["E_a_GVm"], c["U_H_eV_reading"])


@pytest.mark.gpu
def test_library_defaults_are_the_printed_constants():
    import torch
    from paper_2202_10647_gb300 import ionize, workloads as W
    c = constants()
    sd = W.nitrogen()
    E = torch.tensor(np.geomspace(50, 5000, 257), dtype=torch.float64, device="cuda")
    a = ionize.rates(ionize.Species(sd.U, sd.l, sd.m), E, 0, 7)
    b = ionize.rates(ionize.Species(sd.U, sd.l, sd.m, constants=(
        c["omega_a_per_s"], c["E_a_GVm"], c["U_H_eV_reading"])), E, 0, 7)
    assert torch.equal(a, b)
