"""The (l, |m|) factor of Eq. 1 on the GPU: species whose states have
orbital quantum numbers up to l = 3 and projections m = +-1, +-2 (the |m|
term of the power 2n* - |m| - 3/2, the 2^|m| |m|! (l - |m|)! divisor of
f(l, m)), in ion_rates and in the FP32 and FP64 steps, against the oracle;
and the alternative orbital-coupling scenario of Sec. 3 (after Fig. 1: the
electrons left in the p shell couple to a five-fold degenerate singlet d,
a singlet s and a triplet s state) as a table swap of the Kr-like ladder."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2202_10647_gb300 import ionize, workloads as W
from test_gpu_step import adversarial, check, gpu_species, oracle_species, run_both

pytestmark = pytest.mark.gpu


def orbital_ladder() -> W.SpeciesData:
    """A Z = 12 synthetic ladder (the potentials of synthetic_ladder(12))
    with l up to 3 and every projection |m| <= l, signs mixed."""
    base = W.synthetic_ladder(12, seed=120)
    l = [3, 3, 3, 3, 2, 2, 2, 1, 1, 0, 2, 3]
    m = [0, 1, -2, 3, -1, 2, 0, -1, 1, 0, -2, 2]
    return W.SpeciesData("orbital12", base.U, l, m)


def singlet_d_krypton() -> W.SpeciesData:
    """The Kr-like ladder with its states 2-6 taken as the components of a
    singlet d state (l = 2, m = -2..2), state 7 as a singlet s and state 8 as
    a triplet s (l = 0), the rest as in the ladder."""
    sd = W.krypton_like()
    l, m = list(sd.l), list(sd.m)
    for k, mm in zip(range(2, 7), (-2, -1, 0, 1, 2)):
        l[k], m[k] = 2, mm
    l[7], m[7], l[8], m[8] = 0, 0, 0, 0
    return W.SpeciesData("Kr-like singlet d", sd.U, l, m)


SPECIES = {"orbital12": orbital_ladder, "singlet_d_kr": singlet_d_krypton}


@pytest.mark.parametrize("model", [ionize.ION_ADK_CYCLE_AVERAGED, ionize.ION_ADK_STATIC])
@pytest.mark.parametrize("dtype,rtol", [(torch.float32, 2e-6), (torch.float64, 1e-12)])
@pytest.mark.parametrize("name", sorted(SPECIES))
def test_rates_with_l_and_m(name, dtype, rtol, model):
    sd = SPECIES[name]()
    assert max(sd.l) >= 2 and any(abs(m) >= 1 for m in sd.m)
    E = torch.tensor(np.exp(np.linspace(math.log(1e-3), math.log(2e5), 4001)), dtype=dtype)
    sp = ionize.Species(sd.U, sd.l, sd.m, rate_model=model)
    osp = oracle.Species(sd.U, sd.l, sd.m, model=model)
    Wg = ionize.rates(sp, E.cuda(), 0, sd.Z).double().cpu().numpy()
    Wo = oracle.rates(osp, E.double().numpy(), 0, sd.Z)
    big = Wo * 0.05 > 1e-30
    rel = np.abs(Wg[big] - Wo[big]) / Wo[big]
    assert rel.max() <= rtol, rel.max()
    assert np.all(np.abs(Wg[~big]) * 0.05 <= 2e-30)
    # every state with l >= 1 or m != 0 below Kr-like's 13th is exercised
    # where its rate matters (W dt > 1e-3 somewhere on the field grid)
    live = (Wo * 0.05 > 1e-3).any(axis=1)
    assert all(live[k] for k in range(min(sd.Z, 13)) if sd.l[k] or sd.m[k])


def test_m_sign_and_table_swap_on_the_gpu():
    """W depends on |m| only, and the singlet-d swap changes exactly the
    swapped states' rates, by the oracle's ratio."""
    sd = singlet_d_krypton()
    base = W.krypton_like()
    E = torch.tensor(np.exp(np.linspace(math.log(50.0), math.log(5e4), 2001)), dtype=torch.float64)
    flip = W.SpeciesData("flip", sd.U, sd.l, [-m for m in sd.m])
    Wa = ionize.rates(gpu_species(sd), E.cuda(), 0, sd.Z).cpu().numpy()
    Wf = ionize.rates(gpu_species(flip), E.cuda(), 0, sd.Z).cpu().numpy()
    assert np.array_equal(Wa, Wf)
    Wb = ionize.rates(gpu_species(base), E.cuda(), 0, sd.Z).cpu().numpy()
    same = [k for k in range(sd.Z) if (sd.l[k], abs(sd.m[k])) == (base.l[k], abs(base.m[k]))]
    diff = [k for k in range(sd.Z) if k not in same]
    assert diff == [2, 3, 4, 5, 6] + ([7] if base.l[7] != 0 else []) + ([8] if base.l[8] != 0 else [])
    assert np.array_equal(Wa[same], Wb[same])
    osp, obase = oracle_species(sd), oracle_species(base)
    Wo = oracle.rates(osp, E.numpy(), 0, sd.Z)
    Wob = oracle.rates(obase, E.numpy(), 0, sd.Z)
    ok = (Wob[diff] * 0.05 > 1e-30) & (Wo[diff] * 0.05 > 1e-30)
    ratio_gpu = Wa[diff][ok] / Wb[diff][ok]
    ratio_or = Wo[diff][ok] / Wob[diff][ok]
    assert np.abs(ratio_gpu / ratio_or - 1).max() <= 1e-12


@pytest.mark.parametrize("flags", [ionize.ION_F32, ionize.ION_F32 | ionize.ION_NO_FP64_FALLBACK,
                                   ionize.ION_F64_PLAIN])
@pytest.mark.parametrize("name", sorted(SPECIES))
def test_step_with_l_and_m(name, flags):
    """Every window width at the bottom, middle and top of the ladder over
    fields from 0 to 1e6 GV/m and at the crossings of two window rates."""
    sd = SPECIES[name]()
    E, N, lo, hi = adversarial(sd, seed=7)
    out, ref = run_both(sd, E, N, lo, hi, flags=flags)
    check(out, ref, lo, hi, flags)
    n = E.numel()
    tot_in = N.double().numpy().sum(0)[:n]
    assert np.abs(out["N"].sum(0)[:n] - tot_in).max() <= (1e-14 if flags & 1 else 1e-6)


@pytest.mark.parametrize("flags", [ionize.ION_F32, ionize.ION_F64_PLAIN])
def test_lognormal_cells_with_l_and_m(flags):
    """The mixed-batch cell recipe (lognormal |E|, widths 2-6) on the
    singlet-d Kr-like table, windows placed by the plain ladder's thresholds."""
    sd = singlet_d_krypton()
    wl = W.ladder_cells(W.krypton_like(), 20000, seed=23, block=64)
    E, N, lo, hi = wl.E, wl.N, wl.lo, wl.hi
    out, ref = run_both(sd, E, N, lo, hi, flags=flags)
    check(out, ref, lo, hi, flags)
