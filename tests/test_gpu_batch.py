"""Batched and served simulations (vfps_batch_* through the C ABI).

A slot's arithmetic does not depend on its neighbours: the same kernel runs
each instance's CTAs with that instance's descriptor, the reductions of an
instance are done in a fixed order by its own last CTA, and nothing is
accumulated across instances.  So a simulation must give bit-identical psi
and CSR-power series alone and in any mix, and every slot must also match
the FP64 oracle within the FP32 tolerance.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1611_05293_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_05293_b300 import vfps
    vfps.lib()
    return vfps


def alone(V, n, spp, S, Pi, nsteps, psi0, beta=1e-2):
    sim = V.Simulation(V.Params(n=n, steps_per_period=spp, beta=beta), psi0)
    sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, Pi, S)
    sim.step(nsteps)
    out = sim.get_state(), sim.csr_power()
    sim.close()
    return out


def test_lower_order_slots_equal_solo_runs_bitwise(V):
    """N_I = 2, 3 and 4 slots, clamped and not, of several grid sizes and both
    rotations in one batch (launch groups by interpolation order and clamp):
    each equals its solo run."""
    mix = [(64, 500, 0.9, 2.0, 150, 3, 0, 0), (128, 700, 1.2, 1.0, 120, 3, 0, 0), (64, 500, 0.9, 2.0, 150, 4, 0, 0),
           (96, 600, 0.7, 2.0, 90, 2, 0, 0), (64, 400, 0.8, 2.0, 110, 3, 1, 0), (64, 500, 0.9, 2.0, 150, 4, 0, 1),
           (64, 400, 0.8, 2.0, 110, 3, 1, 1)]
    b = V.Batch(len(mix))
    slots = []
    for i, (n, spp, S, Pi, ns, ni, rot, cl) in enumerate(mix):
        slots.append(b.add(V.Params(n=n, steps_per_period=spp, beta=1e-2, interp_points=ni, rotation=rot, clamp=cl),
                           W.blobs(n, 300 + i), V.IMPEDANCE_PARALLEL_PLATES, Pi, S, nsteps=ns))
    b.run(10_000)
    res = [b.take(s) for s in slots]
    b.close()
    for i, (n, spp, S, Pi, ns, ni, rot, cl) in enumerate(mix):
        sim = V.Simulation(V.Params(n=n, steps_per_period=spp, beta=1e-2, interp_points=ni, rotation=rot, clamp=cl),
                           W.blobs(n, 300 + i))
        sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, Pi, S)
        sim.step(ns)
        assert np.array_equal(res[i]["psi"], sim.get_state()), i
        assert np.array_equal(res[i]["power"], sim.csr_power()), i
        sim.close()
    # the orders differ: slot 0 (N_I = 3) and slot 2 (N_I = 4) share everything else
    assert not np.array_equal(res[0]["psi"], res[2]["psi"])


@pytest.mark.parametrize("n,spp", [(1024, 4000), (512, 2000)])
def test_large_grid_shapes_and_solo_give_the_same_bits(V, n, spp):
    """N=512 and 1024 (two warps per column, the column sum as its lower plus
    upper half): batches pinned to CTA widths 8, 4 and 2 and the lone
    simulation (persistent launches) give the same bits; a step matches the
    oracle."""
    ns = 12
    pts = [(0.9, 2.0), (3.0, 1.0), (1.5, 3.0)]
    res = {}
    for W_ in (8, 4, 2):
        b = V.Batch(len(pts))
        b.pin_shape(W_, 1)
        sl = [b.add(V.Params(n=n, steps_per_period=spp, beta=1e-2), W.noisy_gaussian(n, 1614 + i, 1e-6),
                    V.IMPEDANCE_PARALLEL_PLATES, Pi, S, nsteps=ns) for i, (S, Pi) in enumerate(pts)]
        b.run(ns)
        res[W_] = [b.take(s_) for s_ in sl]
        b.close()
    for i, (S, Pi) in enumerate(pts):
        sim = V.Simulation(V.Params(n=n, steps_per_period=spp, beta=1e-2), W.noisy_gaussian(n, 1614 + i, 1e-6))
        sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, Pi, S)
        sim.step(ns)
        psi, P = sim.get_state(), sim.csr_power()
        sim.close()
        for W_ in (8, 4, 2):
            assert np.array_equal(res[W_][i]["psi"], psi), (W_, i)
            assert np.array_equal(res[W_][i]["power"], P), (W_, i)
    op = O.Params(n=n, steps_per_period=spp, beta=1e-2, s_csr=pts[0][0])
    zr, zi = O.impedance(op, 2, pts[0][1])
    ref, Pref, _ = O.run(op, zr, zi, O.normalize(op, W.noisy_gaussian(n, 1614, 1e-6)), 2)
    b = V.Batch(1)
    s0 = b.add(V.Params(n=n, steps_per_period=spp, beta=1e-2), W.noisy_gaussian(n, 1614, 1e-6),
               V.IMPEDANCE_PARALLEL_PLATES, pts[0][1], pts[0][0], nsteps=2)
    b.run(2)
    r = b.take(s0)
    b.close()
    assert np.max(np.abs(r["psi"] - ref)) <= 1e-5 * np.max(np.abs(ref))
    assert np.max(np.abs(r["power"] - Pref)) <= 1e-5 * np.max(np.abs(Pref))


def test_maximum_size_slots_equal_solo_runs(V):
    """n = 2048 (the largest grid): batch slots pinned to CTA widths 4 and 2
    equal the solo run bit for bit."""
    n, spp, ns = 2048, 4000, 6
    ref = None
    sim = V.Simulation(V.Params(n=n, steps_per_period=spp, beta=1e-2), W.noisy_gaussian(n, 7, 1e-3))
    sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, 2.0, 1.5)
    sim.step(ns)
    ref = (sim.get_state(), sim.csr_power())
    sim.close()
    for W_ in (4, 2):
        b = V.Batch(2)
        b.pin_shape(W_, 1)
        sl = [b.add(V.Params(n=n, steps_per_period=spp, beta=1e-2), W.noisy_gaussian(n, 7, 1e-3),
                    V.IMPEDANCE_PARALLEL_PLATES, 2.0, 1.5, nsteps=ns) for _ in range(2)]
        b.run(ns)
        for s_ in sl:
            r = b.take(s_)
            assert np.array_equal(r["psi"], ref[0]) and np.array_equal(r["power"], ref[1]), W_
        b.close()


def test_slot_results_equal_solo_runs_bitwise(V):
    mix = [(64, 500, 0.9, 2.0, 300), (100, 700, 1.2, 1.0, 170), (128, 1000, 0.5, 3.0, 250),
           (64, 500, 0.9, 2.0, 300), (64, 800, 1.7, 2.0, 120), (40, 400, 0.3, 0.5, 90)]
    b = V.Batch(len(mix))
    slots = []
    for i, (n, spp, S, Pi, ns) in enumerate(mix):
        psi0 = W.blobs(n, 100 + (i if i != 3 else 0))
        slots.append(b.add(V.Params(n=n, steps_per_period=spp, beta=1e-2), psi0,
                           V.IMPEDANCE_PARALLEL_PLATES, Pi, S, nsteps=ns))
    b.run(10_000)
    assert sorted(b.poll()) == sorted(slots)
    res = [b.take(s) for s in slots]
    for i, (n, spp, S, Pi, ns) in enumerate(mix):
        assert res[i]["steps"] == ns
        assert res[i]["power"].shape == (ns,)
        psi_a, p_a = alone(V, n, spp, S, Pi, ns, W.blobs(n, 100 + (i if i != 3 else 0)))
        assert np.array_equal(res[i]["psi"], psi_a), i
        assert np.array_equal(res[i]["power"], p_a), i
    # in-batch duplicate (slots 0 and 3): identical inputs, identical outputs
    assert np.array_equal(res[0]["psi"], res[3]["psi"])
    b.close()


def test_slots_match_oracle(V):
    pts = [(48, 500, 0.8, 2.0, 60), (33, 300, 1.4, 1.0, 45)]
    b = V.Batch(4)
    slots = []
    for n, spp, S, Pi, ns in pts:
        slots.append(b.add(V.Params(n=n, steps_per_period=spp, beta=2e-2), W.blobs(n, 7),
                           V.IMPEDANCE_PARALLEL_PLATES, Pi, S, nsteps=ns))
    b.run(1000)
    for s, (n, spp, S, Pi, ns) in zip(slots, pts):
        op = O.Params(n=n, steps_per_period=spp, beta=2e-2, s_csr=S)
        zr, zi = O.impedance(op, 2, Pi)
        ref, pref, _ = O.run(op, zr, zi, O.normalize(op, W.blobs(n, 7)), ns)
        r = b.take(s)
        assert np.max(np.abs(r["psi"] - ref)) / ref.max() < 1e-4
        assert np.max(np.abs(r["power"] - pref) / pref) < 1e-4
    b.close()


def test_budget_admission_and_reuse(V):
    p = V.Params(n=64, steps_per_period=500, beta=1e-2)
    one = V.Batch.slot_bytes(p)
    assert one > 0
    b = V.Batch(4, budget_bytes=one + one // 2)
    s0 = b.add(p, None, V.IMPEDANCE_FREE_SPACE, 0.0, 0.5, nsteps=10)
    assert b.try_add(p, None, V.IMPEDANCE_FREE_SPACE, 0.0, 0.5, nsteps=10) is None   # over budget
    b.run(100)
    assert b.poll() == [s0]
    b.remove(s0)
    assert b.usage() == (0, 0)
    s1 = b.add(p, None, V.IMPEDANCE_FREE_SPACE, 0.0, 0.5, nsteps=10)
    assert s1 == s0
    b.close()
    small = V.Batch(1)
    small.add(p, None, 0, 0.0, 0.0, nsteps=1)
    assert small.try_add(p, None, 0, 0.0, 0.0, nsteps=1) is None                     # no free slot
    small.close()


def test_served_stream_results_equal_solo_runs(V):
    """Continuous batching: requests arrive while others run, are admitted as
    slots free up (3 slots for 10 requests), and each result is the same as
    the request run alone."""
    from paper_1611_05293_b300.serve import Server
    reqs = W.request_stream(10, rate_per_s=1e9, seed=1613, sizes=(32, 48, 64),
                            steps_range=(200, 400), periods_range=(1, 2))
    srv = Server(max_slots=3, chunk_steps=150, beta=1e-2)
    stats = srv.run(reqs, psi0_for=lambda r: W.blobs(r.n, r.rid), realtime=False)
    srv.close()
    assert len(stats.results) == len(reqs)
    assert stats.max_active == 3 and stats.max_queue >= 7
    by_id = {r.rid: r for r in stats.results}
    for q in reqs:
        r = by_id[q.rid]
        assert r.steps == q.nsteps
        psi_a, p_a = alone(V, q.n, q.steps_per_period, q.s_csr, q.Pi, q.nsteps, W.blobs(q.n, q.rid))
        assert np.array_equal(r.psi, psi_a)
        assert np.array_equal(r.power, p_a)
    s = stats.summary()
    assert s["p99_s"] >= s["p50_s"] > 0 and s["cell_updates_per_s"] > 0


def test_large_batch_uses_strips_and_matches_solo_runs(V):
    """256 instances of N=256 (two launch groups of 128): the FP32 streaming
    kernel then walks strips of
    several tiles per CTA (column ring in shared memory); each slot must still
    equal its solo run bit for bit."""
    n, spp, steps = 256, 1000, 3
    pts = W.scan_grid()
    b = V.Batch(256)
    slots = []
    for i in range(256):
        S, Pi = pts[i % len(pts)]
        slots.append(b.add(V.Params(n=n, steps_per_period=spp, beta=1e-2), W.noisy_gaussian(n, 1612 + i % 3),
                           V.IMPEDANCE_PARALLEL_PLATES, Pi, S, nsteps=steps))
    b.run(steps)
    for i in (0, 37, 255):
        S, Pi = pts[i % len(pts)]
        r = b.take(slots[i])
        psi_a, p_a = alone(V, n, spp, S, Pi, steps, W.noisy_gaussian(n, 1612 + i % 3))
        assert np.array_equal(r["psi"], psi_a), i
        assert np.array_equal(r["power"], p_a), i
    b.close()


def test_mixed_rotation_modes_in_one_batch(V):
    """Standard and Manhattan simulations of the same grid size share a batch;
    each slot equals its solo run bit for bit."""
    n, spp, ns = 64, 500, 40
    mix = [(0, 0.9, 2.0), (1, 0.9, 2.0), (1, 1.3, 1.0), (0, 0.5, 3.0)]
    b = V.Batch(len(mix))
    slots = []
    for i, (rot, S, Pi) in enumerate(mix):
        slots.append(b.add(V.Params(n=n, steps_per_period=spp, beta=1e-2, rotation=rot), W.blobs(n, 50 + i),
                           V.IMPEDANCE_PARALLEL_PLATES, Pi, S, nsteps=ns))
    b.run(ns)
    for i, (rot, S, Pi) in enumerate(mix):
        r = b.take(slots[i])
        sim = V.Simulation(V.Params(n=n, steps_per_period=spp, beta=1e-2, rotation=rot), W.blobs(n, 50 + i))
        sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, Pi, S)
        sim.step(ns)
        assert np.array_equal(r["psi"], sim.get_state()), i
        assert np.array_equal(r["power"], sim.csr_power()), i
        sim.close()
    b.close()


def test_batch_moments_equal_solo(V):
    """vfps_batch_moments of a slot equals vfps_moments of the same run alone."""
    n, spp, ns = 128, 800, 30
    b = V.Batch(3)
    slots = [b.add(V.Params(n=n, steps_per_period=spp, beta=1e-2), W.blobs(n, 70 + i),
                   V.IMPEDANCE_PARALLEL_PLATES, 2.0, 0.6 + 0.2 * i, nsteps=ns) for i in range(3)]
    b.run(ns)
    for i, sl in enumerate(slots):
        sim = V.Simulation(V.Params(n=n, steps_per_period=spp, beta=1e-2), W.blobs(n, 70 + i))
        sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, 2.0, 0.6 + 0.2 * i)
        sim.step(ns)
        assert np.array_equal(b.moments(sl), sim.moments()), i
        sim.close()
    b.close()


def test_autotuner_times_candidates_and_keeps_bits(V):
    """The autotuner times candidate launch shapes on the batch's first steps;
    the shapes become final, and results equal the same run with the
    autotuner off (and the solo runs) bit for bit."""
    n, spp, ns, count = 128, 700, 80, 12
    pts = [(0.5 + 0.1 * i, 1.0 + (i % 3)) for i in range(count)]
    out = {}
    for on in (True, False):
        b = V.Batch(count)
        b.autotune(on)
        slots = [b.add(V.Params(n=n, steps_per_period=spp, beta=1e-2), W.blobs(n, 90 + i),
                       V.IMPEDANCE_PARALLEL_PLATES, Pi, S, nsteps=ns) for i, (S, Pi) in enumerate(pts)]
        b.run(ns // 2)
        sh = b.shapes()
        assert sh and all(g["n"] == n for g in sh)
        b.run(ns - ns // 2)
        out[on] = [b.take(s) for s in slots]
        b.close()
    for a, c in zip(out[True], out[False]):
        assert np.array_equal(a["psi"], c["psi"]) and np.array_equal(a["power"], c["power"])


def test_bench_configuration_sampled_slots_match_oracle(V):
    """The benchmark's own launch configuration -- 512 instances of N=256 of
    the parallel-plates scan in one batch, launch shape W=4 with 8-tile strips
    (the autotuner's choice in the timed run), plus the autotuned shape --
    against the FP64 oracle, element by element on sampled slots after two
    steps: relative L-inf <= 1e-5 per step."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    n, spp, beta, steps = 256, 1000, 1e-2, 2
    pts = bench.scan_points(512)
    psi0 = W.noisy_gaussian(n, 1612, 1e-6)
    for pin in ((4, 8), None):
        b = V.Batch(512)
        if pin:
            b.pin_shape(*pin)
        slots = [b.add(V.Params(n=n, steps_per_period=spp, beta=beta), psi0, V.IMPEDANCE_PARALLEL_PLATES, Pi, S,
                       nsteps=steps) for S, Pi in pts]
        b.run(steps)
        if pin:
            assert all(g["W"] == pin[0] and g["tps"] == pin[1] for g in b.shapes() if g["n"] == n)
        for i in (0, 137, 511):
            S, Pi = pts[i]
            op = O.Params(n=n, steps_per_period=spp, beta=beta, s_csr=S)
            zr, zi = O.impedance(op, 2, Pi)
            ref, pref, _ = O.run(op, zr, zi, O.normalize(op, psi0), steps)
            r = b.take(slots[i])
            assert np.max(np.abs(r["psi"] - ref)) / ref.max() < 1e-5 * steps, i
            assert np.max(np.abs(r["power"] - pref) / pref) < 1e-5 * steps, i
        b.close()


def test_pairing_keeps_bits(V):
    """Simulations of equal geometry run two at a time in the pair kernel
    (packed FP32x2); every slot gives the same bits with pairing on and off.
    The mix has an odd one out, two geometries, strong kicks (shifts beyond 4
    cells and shifts that differ by more than one between partners) and
    columns whose y-node is not uniform (per-cell rotation path)."""
    mix = [(64, 100, 12.0, 1.0), (64, 100, 0.9, 2.0), (64, 100, 30.0, 0.5), (64, 100, 0.3, 3.0),
           (64, 100, 2.0, 1.0), (96, 500, 0.9, 2.0), (96, 500, 1.4, 1.0), (256, 1000, 0.8, 2.0),
           (256, 1000, 1.2, 3.0)]
    ns = 6
    out = {}
    for on in (True, False):
        b = V.Batch(len(mix))
        b.pairing(on)
        slots = [b.add(V.Params(n=n, steps_per_period=spp, beta=1e-2), W.blobs(n, 300 + i),
                       V.IMPEDANCE_PARALLEL_PLATES, Pi, S, nsteps=ns) for i, (n, spp, S, Pi) in enumerate(mix)]
        b.run(1)
        sh = b.shapes()
        paired = sum(g["instances"] for g in sh if g["paired"])
        assert paired == (8 if on else 0), sh
        b.run(ns - 1)
        out[on] = [b.take(s) for s in slots]
        b.close()
    for i, (a, c) in enumerate(zip(out[True], out[False])):
        assert np.all(np.isfinite(a["psi"])), i
        assert np.array_equal(a["psi"], c["psi"]), i
        assert np.array_equal(a["power"], c["power"]), i


def test_balanced_grid_keeps_bits(V):
    """The balanced grid (one resident wave of CTAs, each walking an equal
    run of tiles across simulation boundaries, tps = -1) gives the same bits
    as strips of one simulation per CTA, for single and paired simulations."""
    n, spp, ns, count = 256, 1000, 3, 64
    pts = W.scan_grid()
    res = {}
    for shape in ((4, 8), (4, -1), (2, -1), (8, -1)):
        for pair in (False, True):
            b = V.Batch(count)
            b.pin_shape(*shape)
            b.pairing(pair)
            slots = [b.add(V.Params(n=n, steps_per_period=spp, beta=1e-2), W.noisy_gaussian(n, 1612 + i % 3),
                           V.IMPEDANCE_PARALLEL_PLATES, pts[i % len(pts)][1], pts[i % len(pts)][0], nsteps=ns)
                     for i in range(count)]
            b.run(1)
            sh = b.shapes()
            assert all(g["tps"] == shape[1] for g in sh if g["W"] == shape[0]), sh
            b.run(ns - 1)
            res[(shape, pair)] = [b.take(s) for s in slots]
            b.close()
    ref = res[((4, 8), False)]
    for key, r in res.items():
        for i in range(count):
            assert np.array_equal(r[i]["psi"], ref[i]["psi"]), (key, i)
            assert np.array_equal(r[i]["power"], ref[i]["power"]), (key, i)


def test_take_into_preallocated_rows_and_series_bound(V):
    """Batch.take with psi_out (rows of one array) returns the same state as
    a fresh array; the P(t) series is complete whether the slot's target is
    reached or far away (the binding sizes its series buffer by the steps a
    slot can have taken), and a wrong psi_out is refused."""
    n, spp = 48, 400
    b = V.Batch(3)
    slots = [b.add(V.Params(n=n, steps_per_period=spp, beta=1e-2), W.blobs(n, 7 + i),
                   V.IMPEDANCE_PARALLEL_PLATES, 2.0, 0.6, nsteps=ns) for i, ns in enumerate((50, 1 << 40, 80))]
    b.run(30)
    b.run(40)
    rows = np.empty((3, n, n))
    got = [b.take(s, psi_out=rows[i]) for i, s in enumerate(slots)]
    ref = [b.take(s) for s in slots]
    for i, ns in enumerate((50, 70, 70)):
        assert got[i]["steps"] == ns and got[i]["power"].shape == (ns,), i
        assert got[i]["psi"] is rows[i] or np.shares_memory(got[i]["psi"], rows)
        assert np.array_equal(rows[i], ref[i]["psi"]), i
        assert np.array_equal(got[i]["power"], ref[i]["power"]), i
    with pytest.raises(ValueError):
        b.take(slots[0], psi_out=np.empty((n, n), dtype=np.float32))
    with pytest.raises(ValueError):
        b.take(slots[0], psi_out=np.empty((n, n + 1)))
    b.close()


def test_bulk_add_and_take_equal_single_calls(V):
    """vfps_batch_add_many / vfps_batch_take_many move many slots in one copy
    each way (normalisation and FP32 conversion on the device) and give the
    same bits as one vfps_batch_add / vfps_batch_take per slot; a bad state
    anywhere refuses the whole call and adds nothing."""
    n, spp, steps = 64, 500, 40
    pts = [(0.3, 2.0), (0.9, 1.0), (1.4, 3.0), (0.6, 0.5), (1.1, 2.5)]
    psi0 = np.stack([W.blobs(n, 40 + i) for i in range(len(pts))])
    params = V.Params(n=n, steps_per_period=spp, beta=1e-2)
    one = V.Batch(len(pts))
    s1 = [one.add(params, psi0[i], V.IMPEDANCE_PARALLEL_PLATES, Pi, S, nsteps=steps) for i, (S, Pi) in enumerate(pts)]
    one.run(steps)
    ref = [one.take(sl) for sl in s1]
    one.close()
    many = V.Batch(len(pts) + 2)
    bad = psi0.copy()
    bad[3, 5, 5] = np.inf
    with pytest.raises(V.VfpsError) as e:
        many.add_many(params, bad, V.IMPEDANCE_PARALLEL_PLATES, [p[1] for p in pts], [p[0] for p in pts], steps)
    assert e.value.code == V.EINVAL and many.usage()[0] == 0
    sm = many.add_many(params, psi0, V.IMPEDANCE_PARALLEL_PLATES, [p[1] for p in pts], [p[0] for p in pts], steps)
    many.run(steps)
    out = np.empty((len(pts), n, n))
    power = many.take_many(sm, psi_out=out, power_cap=steps)
    for i in range(len(pts)):
        assert np.array_equal(out[i], ref[i]["psi"]), i
        assert np.array_equal(power[i], ref[i]["power"]), i
        assert np.array_equal(many.take(sm[i])["psi"], ref[i]["psi"]), i
    many.close()


def test_bulk_edges_and_mixed_precision(V):
    """vfps_batch_add_many refuses a request larger than the free slots
    (EBUSY, nothing added); vfps_batch_take_many gathers FP32 and FP64 slots
    of different grid sizes in one call, each equal to its own take."""
    p32 = V.Params(n=48, steps_per_period=300, beta=1e-2)
    p64 = V.Params(n=48, steps_per_period=300, beta=1e-2, precision=1)
    b = V.Batch(4)
    with pytest.raises(V.VfpsError) as e:
        b.add_many(p32, None, V.IMPEDANCE_FREE_SPACE, [0.0] * 5, [0.4] * 5, 10)
    assert e.value.code == V.EBUSY and b.usage()[0] == 0
    s32 = b.add_many(p32, None, V.IMPEDANCE_FREE_SPACE, [0.0, 0.0], [0.4, 0.8], 25)
    s64 = b.add_many(p64, None, V.IMPEDANCE_FREE_SPACE, [0.0], [0.6], 25)
    b.run(25)
    slots = s32 + s64
    out = np.empty((3, 48, 48))
    power = b.take_many(slots, psi_out=out, power_cap=25)
    for i, sl in enumerate(slots):
        r = b.take(sl)
        assert np.array_equal(out[i], r["psi"]) and np.array_equal(power[i], r["power"]), sl
    b.close()


def test_recording_slot_leaves_the_pair_kernel(V):
    """With pairing on, a slot that records moments runs in the single-
    simulation kernel (the pair kernel has no moment pass) and both slots
    keep the bits of their solo runs."""
    n, spp = 64, 500
    params = V.Params(n=n, steps_per_period=spp, beta=1e-2)
    b = V.Batch(2)
    b.pairing(True)
    sa = b.add(params, None, V.IMPEDANCE_PARALLEL_PLATES, 2.0, 0.9, nsteps=40)
    sb = b.add(params, None, V.IMPEDANCE_PARALLEL_PLATES, 2.0, 1.1, nsteps=40)
    b.record_moments(sb, 8)
    b.run(1)
    assert not any(g["paired"] for g in b.shapes())
    b.run(39)
    got = {sa: b.take(sa), sb: b.take(sb)}
    rec = b.moment_series(sb)
    b.close()
    assert rec.shape == (5, 5)
    for sl, S in ((sa, 0.9), (sb, 1.1)):
        psi_a, p_a = alone(V, n, spp, S, 2.0, 40, None)
        assert np.array_equal(got[sl]["psi"], psi_a) and np.array_equal(got[sl]["power"], p_a)


def test_spectrogram_rejects_bad_windows(V):
    sim = V.Simulation(V.Params(n=32, steps_per_period=200, beta=1e-2), None)
    sim.set_impedance(V.IMPEDANCE_FREE_SPACE, 0.0, 0.5)
    sim.step(300)
    for L, hop, count in ((100, 10, 2), (256, 0, 2), (256, 16, 0), (256, 64, 2)):  # not 2^k, hop, count, span
        with pytest.raises(V.VfpsError) as e:
            sim.spectrogram(L, hop, count)
        assert e.value.code == V.EINVAL, (L, hop, count)
    assert sim.spectrogram(256, 44, 2).shape == (2, 129)
    sim.close()
