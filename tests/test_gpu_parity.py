"""Parity of the CUDA library with the FP64 oracle on the same seeded problems.

FP64 particle records: cell indices, the stable per-cell order (the sort permutation) and the
per-cell NTC candidate / accepted-pair, absorption and re-sampling counts bit-exact over 20
steps; particle state and the total state Psi_t within 1e-9 relative (the two sides differ only
in the rounding order of sums and in last-bit differences of library transcendentals).
FP32 particle records: the oracle stores the particle state in single precision at the same
points and takes the transport decision in single precision (one fused multiply-add), so the
same decisions are taken; per-particle state within 1e-5 relative over 5 steps.
"""
import numpy as np
import pytest

import oracle as O
from paper_2305_12071_gb300 import workloads as W
from parity_util import compare_counters, compare_fields, compare_particles, solver

pytestmark = pytest.mark.gpu

REL64 = 1e-9
REL32 = 1e-5


def _run_pair(params, checkpoints, rel_p, rel_f, counters=True):
    g = solver(params)
    o = O.Oracle(params)
    done = 0
    for n in checkpoints:
        g.step(n - done)
        o.step(n - done)
        done = n
        what = f"step {n}"
        compare_particles(g.particles(), o.particles(), rel_p, what)
        compare_fields(g.fields()[0], o.psi(), rel_f, what)
        if counters:
            compare_counters(g.counters(), o.counters(), what)
        # c_max is raised to a candidate pair's relative speed (Appendix A), computed from particle
        # velocities that agree to rel_p: it agrees to the same relative tolerance
        assert np.allclose(g.cmax(), o.cmax(), rtol=rel_p, atol=0), what
    g.close()


def test_shock_mach3_fp64_20_steps():
    _run_pair(W.config1("fp64"), [1, 2, 5, 20], REL64, REL64)


def test_shock_mach3_fp32_5_steps():
    _run_pair(W.config1("fp32"), [1, 2, 5], REL32, REL64)


@pytest.mark.parametrize("Kn", [1e-4, 1e-3])
def test_sod_wave_regime_fp64(Kn):
    # P > 0: absorption, re-sampling and the NS wave flux are all active
    p = W.sod(n_cells=120, Kn=Kn, ppc_ref=150, precision="fp64", seed=7)
    _run_pair(p, [1, 3, 20], REL64, REL64)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_dense_shock_block_kernel_hashed(precision):
    # P = 0 cells with 100-400 NTC candidates among 1000-2400 particles: the block kernel on lists
    # longer than its table, the touched particles of each window hashed
    p = W.shock(8.0, omega=0.81, n_cells=60, ppc_ref=600.0, precision=precision, seed=11)
    if precision == "fp64":
        _run_pair(p, [1, 3, 10], REL64, REL64)
    else:
        _run_pair(p, [1, 3], REL32, REL64)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_staged_rounds_with_cmax_raises(precision):
    # a Mach-8 shock at small Kn: every cell absorbs (P > 0, staged lists collided in dependency
    # rounds on one warp), and hot particles meeting cold cells raise c_max inside a batch (the
    # oracle finds such raises in light staged cells over these steps), so the rerun of a batch up
    # to its raising candidate is exercised
    p = W.shock(8.0, omega=0.81, n_cells=80, ppc_ref=60.0, precision=precision, seed=3)
    p["Kn"] = 0.01
    o = O.Oracle(p)
    raised = 0
    for _ in range(10):
        cm0, P = o.cmax().copy(), o.prim()["P"].copy()
        o.step(1)
        raised += int(((o.cmax() > cm0) & (P > 0) & (o.counters()["ncand"] < 96)).sum())
    assert raised > 0
    if precision == "fp64":
        _run_pair(p, [1, 4, 10], REL64, REL64)
    else:
        _run_pair(p, [1, 3, 5], REL32, REL64)


def test_sod_wave_regime_fp32():
    p = W.sod(n_cells=120, Kn=3e-4, ppc_ref=150, precision="fp32", seed=8)
    _run_pair(p, [1, 5], REL32, REL64)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ns_corrected_resampling(precision):
    # resample_mode CE: particles drawn from the wave follow the Maxwellian times its Chapman-Enskog
    # factor (acceptance-rejection, up to 64 attempts); mirror walls give the end cells' neighbours
    p = W.sod(n_cells=120, Kn=3e-4, ppc_ref=150, precision=precision, seed=9, resample_mode="ce")
    if precision == "fp64":
        _run_pair(p, [1, 3, 20], REL64, REL64)
    else:
        _run_pair(p, [1, 5], REL32, REL64)
    # the option is in effect: the first step's samples differ from the plain Maxwellian's
    a, b = solver(p), solver(dict(p, resample_mode="maxwell"))
    a.step(1)
    b.step(1)
    pa, pb = a.particles(), b.particles()
    assert len(pa["u"]) == len(pb["u"])
    assert np.setdiff1d(pa["u"], pb["u"]).size > 20
    a.close()
    b.close()
    # inflow reservoirs beside the end cells (their own samples stay Maxwellian)
    q = dict(W.config1(precision), Kn=2e-3, n_cells=80, ppc_ref=60, resample_mode="ce")
    _run_pair(q, [1, 10] if precision == "fp64" else [1, 4], REL64 if precision == "fp64" else REL32, REL64)


def test_resample_mode_is_validated():
    import ctypes as C
    from paper_2305_12071_gb300 import build as B
    from paper_2305_12071_gb300 import duwp
    B.build()
    L = duwp.load()
    prm = duwp.make_params(dict(W.config1("fp64"), n_cells=20))
    prm.resample_mode = 2
    h = C.c_void_p()
    assert L.duwp_init(C.byref(prm), None, duwp.ALLOC_FN(0), duwp.FREE_FN(0), None, C.byref(h)) == -1
    assert not h.value
    prm = duwp.make_params(dict(W.config1("fp64"), n_cells=20))
    prm.split_mode = 2
    assert L.duwp_init(C.byref(prm), None, duwp.ALLOC_FN(0), duwp.FREE_FN(0), None, C.byref(h)) == -1
    assert not h.value
    prm = duwp.make_params(dict(W.config1("fp64"), n_cells=20))
    prm.recon_mode = 2
    assert L.duwp_init(C.byref(prm), None, duwp.ALLOC_FN(0), duwp.FREE_FN(0), None, C.byref(h)) == -1
    assert not h.value


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_second_order_wave_reconstruction(precision):
    # recon_mode vanleer: limited linear interface states in the wave flux; mirror walls (Sod),
    # a periodic box with a density wave, and inflow reservoirs (a wave-regime shock)
    p = W.sod(n_cells=120, Kn=1e-4, ppc_ref=150, precision=precision, seed=13, recon_mode="vanleer")
    q = W.uniform(n_cells=64, Kn=1e-4, ppc_ref=80, state=(1.0, 0.4, 0.0, 0.0, 1.0), bc="periodic", x_max=1.0,
                  dt=2e-3, precision=precision, seed=14, recon_mode="vanleer", x_split=0.3,
                  left=(1.0, 0.4, 0.0, 0.0, 1.0), right=(0.5, 0.4, 0.0, 0.0, 1.6))
    r = dict(W.config1(precision), Kn=2e-3, n_cells=80, ppc_ref=60, recon_mode="vanleer")
    for case in (p, q, r):
        if precision == "fp64":
            _run_pair(case, [1, 3, 15], REL64, REL64)
        else:
            _run_pair(case, [1, 4], REL32, REL64)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_qmc_split(precision):
    # split_mode qmc (Sec. 3.2/3.3): every usable cell has P = 1 - exp(-dt/tau) > 0 (absorption and
    # re-sampling everywhere) and every interface carries a weighted wave flux
    p = W.sod(n_cells=120, Kn=3e-4, ppc_ref=150, precision=precision, seed=11, split_mode="qmc")
    q = dict(W.config1(precision), split_mode="qmc")   # the Mach-3 shock, where Eq. (p) gives P = 0
    if precision == "fp64":
        _run_pair(p, [1, 3, 20], REL64, REL64)
        _run_pair(q, [1, 5, 12], REL64, REL64)
    else:
        _run_pair(p, [1, 5], REL32, REL64)
        _run_pair(q, [1, 4], REL32, REL64)
    o = O.Oracle(q)
    o.step(2)
    assert np.all(o.prim()["P"] > 0) and o.counters()["nabs"].sum() > 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_periodic_far_movers(precision):
    # a time step of ~1.6 cells at the thermal speed: many particles move two or more cells,
    # and the periodic wrap sends particles across the whole domain
    p = W.uniform(n_cells=37, Kn=0.05, ppc_ref=80, state=(1.0, 0.7, 0.0, 0.0, 1.0), bc="periodic",
                  x_max=1.0, dt=0.02, precision=precision, seed=11)
    o = O.Oracle(p)
    o.step(2)
    assert o.last_nfar() > 50
    _run_pair(p, [1, 2, 8], REL64 if precision == "fp64" else REL32, REL64)


def test_free_expansion_walls_and_vacuum():
    p = W.base(Kn=0.2, n_cells=64, x_min=-1.0, x_max=1.0, left=(1, 0.2, 0, 0, 1), right=(0, 0, 0, 0, 1),
               x_split=0.0, bc_left="specular", bc_right="vacuum", ppc_ref=120, seed=3, precision="fp64")
    _run_pair(p, [1, 4, 20], REL64, REL64)


def test_ragged_small_cases():
    # one cell; two cells; cells with fewer than two particles (no collisions possible)
    for C, ppc in ((1, 50), (2, 3), (5, 1.5)):
        p = W.uniform(n_cells=C, Kn=0.3, ppc_ref=ppc, state=(1.0, 0.1, 0.0, 0.0, 1.0), bc="specular",
                      x_max=1.0, dt=0.05, seed=5)
        _run_pair(p, [1, 6], REL64, REL64)


def test_hard_sphere_and_total_rate_options():
    p = W.config1("fp64")
    p.update(omega=0.5, ntc_rate="total", eps_mode="eps12", n_cells=40, ppc_ref=60)
    _run_pair(p, [1, 10], REL64, REL64)
    p = W.sod(n_cells=80, Kn=2e-4, ppc_ref=60, precision="fp64", flux_mode="kfvs", eps_mode="eps_avg", seed=4)
    _run_pair(p, [1, 10], REL64, REL64)


def test_batch_equals_alone():
    ps = [W.config1("fp64"), W.sod(n_cells=90, Kn=1e-3, ppc_ref=100, seed=9),
          W.uniform(n_cells=17, bc="periodic", dt=0.02, x_max=1.0, ppc_ref=60, seed=2)]
    b = solver(ps)
    b.step(7)
    for i, p in enumerate(ps):
        a = solver(p)
        a.step(7)
        pa, pb = a.particles(), b.particles(i)
        for k in pa:
            assert np.array_equal(pa[k], pb[k]), f"instance {i} field {k}"
        assert np.array_equal(a.fields()[0], b.fields(i)[0])
        a.close()
    b.close()


def test_large_pool_cell_blocks_change_no_result():
    # past 2 x 128 x SMs flattened cells the cell kernel runs in smaller blocks than the offset
    # kernel (which then reads several of its block sums per block): the small instances of such a
    # batch (a ragged cell count) must equal the same instances alone, where both kernels share one
    # block size
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    big = W.uniform(n_cells=2 * 128 * nsm + 777, ppc_ref=4, precision="fp32", seed=21)
    ps = [W.sod(n_cells=90, Kn=1e-3, ppc_ref=100, precision="fp32", seed=9), big, W.config1("fp32")]
    b = solver(ps)
    b.step(6)
    for i in (0, 2):
        a = solver(ps[i])
        a.step(6)
        pa, pb = a.particles(), b.particles(i)
        for k in pa:
            assert np.array_equal(pa[k], pb[k]), f"instance {i} field {k}"
        assert np.array_equal(a.fields()[0], b.fields(i)[0])
        a.close()
    b.close()


def test_graphs_and_plain_launches_agree():
    p = W.sod(n_cells=100, Kn=1e-3, ppc_ref=100, precision="fp32", seed=12)
    a = solver(p, graphs=True)
    b = solver(p, graphs=False)
    a.step(9)
    b.step(9)
    pa, pb = a.particles(), b.particles()
    for k in pa:
        assert np.array_equal(pa[k], pb[k])
    assert np.array_equal(a.fields()[0], b.fields()[0])


def test_checkpoint_resume_bit_exact():
    p = W.config1("fp32")
    a = solver(p)
    a.step(10)
    blob = a.checkpoint()
    a.step(10)
    b = solver(p)
    b.restore(blob)
    b.step(10)
    pa, pb = a.particles(), b.particles()
    for k in pa:
        assert np.array_equal(pa[k], pb[k])
    assert np.array_equal(a.fields()[0], b.fields()[0])


def test_time_average_matches_oracle():
    p = W.config1("fp64")
    p["avg_start"] = 5
    g = solver(p)
    o = O.Oracle(p)
    g.step(12)
    o.step(12)
    ga, gn = g.fields(which=1)
    oa, on = o.avg()
    assert gn == on == 7
    compare_fields(ga, oa, REL64)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_launch_shape_does_not_change_results(precision):
    # threads per block (warps per block), the register budget and the record groups per lane
    p = W.sod(n_cells=120, Kn=3e-4, ppc_ref=150, precision=precision, seed=8)
    ref = None
    for t, r, g in ((128, 0, 2), (32, 0, 2), (256, 0, 3), (512, 0, 2), (128, 1, 3), (512, 1, 2), (64, 2, 3),
                    (512, 2, 2), (256, 1, 3)):
        s = solver(p)
        s.set_launch(t, r, g)
        s.step(6)
        got = (s.particles(), s.fields()[0], s.counters())
        s.close()
        if ref is None:
            ref = got
            continue
        for k in ref[0]:
            assert np.array_equal(ref[0][k], got[0][k]), f"{t}/{r}/{g}: particles {k}"
        assert np.array_equal(ref[1], got[1]), f"{t}/{r}/{g}: fields"
        for k in ref[2]:
            assert np.array_equal(ref[2][k], got[2][k]), f"{t}/{r}/{g}: counter {k}"


def test_moments_all_equals_per_instance():
    ps = [W.config1("fp32"), W.sod(n_cells=90, Kn=1e-3, ppc_ref=100, precision="fp32", seed=9),
          W.uniform(n_cells=17, bc="periodic", dt=0.02, x_max=1.0, ppc_ref=60, seed=2, precision="fp32")]
    for p in ps:
        p["avg_start"] = 2
    g = solver(ps)
    g.step(6)
    for which in (0, 1):
        allm = g.moments_all(which)
        o = 0
        for i in range(g.n):
            m = g.moments(i, which)
            n = g.n_cells(i)
            for k in m:
                assert np.array_equal(allm[k][o:o + n], m[k]), f"instance {i} {k} which {which}"
            o += n
    g.close()


def test_async_moments_equal_synchronous_reads():
    # reads enqueued behind each step into pinned arrays, overlapping the next step's kernels, equal
    # the synchronous reads of a twin run bit for bit (three or more reads in flight exercise the
    # reuse of the two device areas)
    import torch
    plist = [W.shock(m, n_cells=n, ppc_ref=80, precision="fp32", seed=30 + k)
             for k, (m, n) in enumerate(((2.0, 70), (5.0, 130), (3.0, 41)))]
    a, b = solver(plist), solver(plist)
    total = sum(int(p["n_cells"]) for p in plist)
    bufs = [{k: torch.empty(total, dtype=torch.float64, pin_memory=True).numpy() for k in ("rho", "u", "T", "wave_frac")}
            for _ in range(6)]
    for j in range(6):
        a.step(1)
        a.moments_all_async(bufs[j])
    a.moments_wait()
    for j in range(6):
        b.step(1)
        ref = b.moments_all()
        for k in ref:
            assert np.array_equal(ref[k], bufs[j][k]), (j, k)
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_overlapped_step_equals_serial_step(precision):
    # duwp_step streams the cells that need nothing from the collision kernel on a side stream while
    # it runs; duwp_step_timed runs the kernels one after the other: same particles and states
    plist = [W.shock(m, n_cells=n, ppc_ref=70, precision=precision, seed=40 + k)
             for k, (m, n) in enumerate(((1.5, 60), (6.0, 150), (3.0, 90)))]
    a, b = solver(plist), solver(plist)
    a.step(6)
    b.step_timed(6)
    for i in range(len(plist)):
        pa, pb = a.particles(i), b.particles(i)
        for k in pa:
            assert np.array_equal(pa[k], pb[k]), (i, k)
        assert np.array_equal(a.fields(i)[0], b.fields(i)[0]), i
    a.close()
    b.close()
