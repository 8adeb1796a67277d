"""The stated number of steps of the two large cavity configurations against
the FP64 oracle (its OpenMP build on all host cores).  The oracle needs about
30 minutes of host time for all three, so these run only with FVGB_LONG=1 (the
default suite compares the first five and the first two steps of the same
configurations, tests/test_gpu_zz_full_configs.py and test_gpu_zz_full8m.py).

* 1M-cell cavity (100^3, seed 1234 permutation, RCM; nu 0.01, dt 0.002):
  all 50 PISO steps, FP64, against the oracle and its own spread under 1e-15
  input perturbations (bar: max(1e-9, 10x that spread) per field, pressure
  split into mean-free part and mean; iteration counts within 1 wherever the
  perturbed oracle runs agree on them).
* 8M-cell cavity (200^3; nu 0.01, dt 0.001): all 20 PISO steps, FP64 and
  mixed precision, each against the FP64 oracle; the FP64 run held to the
  same bar as the 1M run (its first two steps are within 1e-9 in the
  default suite), the mixed run's per-field error reported (``-rA``) and
  bounded by the 1e-6 solver tolerance's reach.
* the SIMPLE channel (2,654,208 jittered tetrahedra): the first 30 SIMPLE
  iterations against the oracle and its spread (the converged run is
  checked against the duct series in test_gpu_channel.py; the whole run,
  about 2,600 iterations, would take the oracle hours).
* the batch of 256 cavities (seed 7): all 200 steps, every case against its
  own oracle run (one sequential oracle per host thread), strict where the
  case's iteration counts agree within 1 and its fields within 1e-9, else
  held to the case's own oracle envelope; where the GPU took a near-threshold
  CG stop that none of the perturbed oracle runs took, the oracle is replayed
  with every pressure solve held to the GPU's iteration count and the fields
  compared with that replay."""
import concurrent.futures as cf
import os
import time

import numpy as np
import pytest

import meshgen as mg
import oracle as O
from parity_util import (TOL, field_errors, oracle_spread, assert_errors_within,
                         assert_iters_where_well_conditioned)

pytestmark = [pytest.mark.gpu, pytest.mark.slow,
              pytest.mark.skipif(os.environ.get("FVGB_LONG") != "1",
                                 reason="long oracle runs: set FVGB_LONG=1")]


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1207_1571_gb300 import build as B
    B.build()
    import paper_1207_1571_gb300 as P
    P.load()
    O.set_threads(os.cpu_count() or 1)
    return P


def test_cavity_100_cubed_all_50_steps(P):
    n, nsteps = 100, 50
    m = mg.permute_cells(mg.cavity3d(n), mg.random_permutation(n ** 3, 1234))
    step = lambda c, k: c.piso_step(0.002, 2, p_ref_cell=m.corner_cell)
    t0 = time.perf_counter()
    base, its0, its_p, spread = oracle_spread(m, 0.01, nsteps, step, parallel=True)
    t_or = time.perf_counter() - t0
    case = P.Case(P.Mesh(m, renumber=True), 0.01)
    gpu_its = [case.piso_step(0.002, 2, p_ref_cell=m.corner_cell)["iters"] for _ in range(nsteps)]
    stable = assert_iters_where_well_conditioned(gpu_its, its0, its_p)
    errs = field_errors(case.get_fields_host(), base.get_fields())
    print(f"\n100^3 cavity, {nsteps} steps: errors {errs}\n oracle spread {spread}\n"
          f" stable solves {int(stable.sum())}/{stable.size}; oracle (3 runs) {t_or:.0f} s")
    assert_errors_within(errs, spread)


def test_cavity_200_cubed_all_20_steps_fp64_and_mixed(P):
    """20 steps are long enough for the tolerance-truncated CG to amplify
    rounding past 1e-9 (as on the 1M cavity after 50 steps), so the FP64 run
    is held to the oracle's own spread under 1e-15 input perturbations
    (three oracle runs)."""
    n, nsteps = 200, 20
    m = mg.permute_cells(mg.cavity3d(n), mg.random_permutation(n ** 3, 1234))
    step = lambda c, k: c.piso_step(0.001, 2, p_ref_cell=m.corner_cell)
    t0 = time.perf_counter()
    base, its0, its_p, spread = oracle_spread(m, 0.01, nsteps, step, parallel=True)
    t_or = time.perf_counter() - t0
    mesh = P.Mesh(m, renumber=True)
    c64 = P.Case(mesh, 0.01)
    cmx = P.Case(mesh, 0.01, P.FV_PREC_MIXED)
    gpu_its = []
    for k in range(nsteps):
        s = c64.piso_step(0.001, 2, p_ref_cell=m.corner_cell)
        sm = cmx.piso_step(0.001, 2, p_ref_cell=m.corner_cell)
        assert s["status"] == 0 and sm["status"] == 0, (k, s, sm)
        assert all(x["res"] <= 1e-6 for x in sm["p"]), (k, sm)
        gpu_its.append(s["iters"])
    stable = assert_iters_where_well_conditioned(gpu_its, its0, its_p)
    ref = base.get_fields()
    e64 = field_errors(c64.get_fields_host(), ref)
    emx = field_errors(cmx.get_fields_host(), ref)
    print(f"\n200^3 cavity, {nsteps} steps: FP64 vs oracle {e64}\n oracle spread {spread}\n"
          f" mixed vs FP64 oracle {emx}\n stable solves {int(stable.sum())}/{stable.size}; "
          f"oracle (3 runs) {t_or:.0f} s")
    assert_errors_within(e64, spread)
    assert emx["u"] < 1e-5 and emx["phi"] < 1e-5 and emx["p_meanfree"] < 1e-4, emx


def test_channel_first_30_simple_iterations(P):
    m = mg.duct_tets(48, 192, jitter=0.1, seed=2024)
    F = m.n_internal_faces
    q = m.patch("inlet")
    inl = m.patches[q]
    prof = mg.duct_inlet_profile(m.Cf[:2, F + inl.start:F + inl.start + inl.size])
    inlet = np.stack([0 * prof, 0 * prof, prof])
    nit = 30

    def step(c, n):
        if n == 0:
            c.set_patch_faces(q, inlet)
        return c.simple_iter(0.7, 0.3)
    t0 = time.perf_counter()
    base, its0, its_p, spread = oracle_spread(m, 0.05, nit, step, parallel=True)
    t_or = time.perf_counter() - t0
    case = P.Case(P.Mesh(m, renumber=True), 0.05)
    case.set_patch_faces(q, inlet)
    gpu_its = [case.simple_iter(0.7, 0.3)["iters"] for _ in range(nit)]
    stable = assert_iters_where_well_conditioned(gpu_its, its0, its_p)
    errs = field_errors(case.get_fields_host(), base.get_fields())
    print(f"\nchannel, {nit} SIMPLE iterations: errors {errs}\n oracle spread {spread}\n"
          f" stable solves {int(stable.sum())}/{stable.size}; oracle (3 runs) {t_or:.0f} s")
    assert_errors_within(errs, spread, keys=("u", "phi", "p"))


def _oracle_batch_case(args):
    """One case's oracle run; with eps > 0 from a rest state perturbed by an
    eps-sized random velocity (the oracle's own rounding sensitivity)."""
    om, m, nu, ref, nsteps, eps, seed = args
    oc = O.Case(om, nu)
    if eps > 0:
        u = np.zeros((3, m.n_cells))
        u[:2] = eps * np.random.default_rng(seed).standard_normal((2, m.n_cells))
        oc.set_fields(u, np.zeros(m.n_cells), np.zeros(m.n_faces))
    its = [np.array(oc.piso_step(0.002, 2, p_ref_cell=ref)["iters"]) for _ in range(nsteps)]
    return np.array(its), oc.get_fields()


def _oracle_replay(args):
    """A case's oracle run with every pressure solve held to the given
    iteration counts (another run's stopping decisions)."""
    om, nu, ref, its = args
    oc = O.Case(om, nu)
    for it in its:
        oc.piso_step(0.002, 2, p_ref_cell=ref, p_iters=np.asarray(it)[3:])
    return oc.get_fields()


def test_batch_all_256_cases_all_200_steps(P):
    nsteps = 200
    spec = mg.batch_cases(256, 7)
    ms = [mg.cavity2d(n) for n, _ in spec]
    nus = [nu for _, nu in spec]
    refs = [m.corner_cell for m in ms]
    bt = P.Batch(ms, nus, refs)
    gpu_its = [[] for _ in ms]
    for _ in range(nsteps):
        st = bt.piso_step(0.002, 2)
        for k in range(len(ms)):
            assert st[k]["status"] == 0, (k, st[k])
            gpu_its[k].append(np.array(st[k]["iters"]))
    gpu = [bt.get_fields(k) for k in range(len(ms))]
    # oracle meshes in this thread (the renumbering is not reentrant), the
    # case runs over the host cores
    oms = [O.Mesh(m, renumber=True) for m in ms]
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        res = list(ex.map(_oracle_batch_case, [(om, m, nu, r, nsteps, 0.0, 0)
                                               for om, m, nu, r in zip(oms, ms, nus, refs)]))
        loose = []
        worst = {q: 0.0 for q in ("u", "phi", "p_meanfree", "p_mean")}
        for k, (its_o, fo) in enumerate(res):
            errs = field_errors(gpu[k], fo)
            for q in worst:
                worst[q] = max(worst[q], errs[q])
            if not (np.abs(np.array(gpu_its[k]) - its_o).max() <= 1
                    and all(errs[q] <= TOL for q in worst)):
                loose.append(k)
        # the cases whose stopping iterations are rounding-decided: against
        # their own oracle envelope (four runs from 1e-15-perturbed rest
        # states; over 200 steps two runs miss some near-threshold stops)
        seeds = (1, 2, 3, 4)
        pert = list(ex.map(_oracle_batch_case, [(oms[k], ms[k], nus[k], refs[k], nsteps, 1e-15, sd)
                                                for k in loose for sd in seeds]))
        ns = len(seeds)
        n_stable, off, spreads, replay = 0, [], {}, []
        for j, k in enumerate(loose):
            its0, f0 = res[k]
            runs = pert[ns * j:ns * (j + 1)]
            spread = {}
            stable = np.ones_like(its0, bool)
            for its, f in runs:
                stable &= its == its0
                for q, v in field_errors(f, f0).items():
                    spread[q] = max(spread.get(q, 0.0), v)
            spreads[k] = spread
            diff = np.abs(np.array(gpu_its[k]) - its0)
            n_stable += int(stable.sum())
            bad = [(k, int(a), int(b), int(diff[a, b])) for a, b in np.argwhere(stable & (diff > 1))]
            off += bad
            errs = field_errors(gpu[k], f0)
            if bad or any(errs[q] > max(TOL, 10 * spread[q]) for q in worst):
                replay.append(k)
        # a case whose GPU run took a near-threshold CG stop the perturbed
        # oracle runs did not take (the GPU's own summation order decides it):
        # the oracle replayed along the GPU's branch -- every pressure solve
        # held to the GPU's iteration count -- must then agree to rounding
        rep = list(ex.map(_oracle_replay, [(oms[k], nus[k], refs[k], gpu_its[k]) for k in replay]))
    for k, fr in zip(replay, rep):
        assert_errors_within(field_errors(gpu[k], fr), spreads[k])
    for k in loose:
        if k not in replay:
            assert_errors_within(field_errors(gpu[k], res[k][1]), spreads[k])
    print(f"\nbatch of 256 cavities, {nsteps} steps: worst errors {worst}; {len(loose)} cases "
          f"held to their oracle envelope ({n_stable} solves with a reproducible count; "
          f"off by more than 1: {off}); replayed along the GPU's stops: {replay}; "
          f"oracle {time.perf_counter() - t0:.0f} s")
