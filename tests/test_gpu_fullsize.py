"""Parity at the benchmark's full size (sparse logistic 200000 x 5000 FP32, N=16, M=8,
kappa=50, rho=0.5) in the launch configuration bench.py times, on outputs the oracle can
compute alone, plus properties that hold at any size.

* After iteration 1, x = 0, so omega_r = prox(0; b_r) for every row (eq. p:GPU;omega).
* After iteration 1, z = u = 0, so iteration 2's x-step of shard 0 depends on shard 0 only:
  the oracle runs that shard alone (with the global N in the ridge coefficient) on the
  FP32-rounded rows and is compared with x_0, omega and nu of shard 0.
* z, s, t, v after iteration 2: the s-step / (z,t) relations checked as properties.
"""
import numpy as np
import pytest

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import bicadmm as bc
from paper_2405_16267_b300 import synth

from gpu_util import check_consensus_step, consensus_state

pytestmark = pytest.mark.gpu

TOL32 = 1e-4


@pytest.fixture(scope="module")
def run():
    import torch
    import bench
    wl = dict(bench.WORKLOAD)
    A, b, _ = bench.generate(wl)
    A_t = torch.from_numpy(A).cuda()
    b_t = torch.from_numpy(b).cuda()
    with bc.Solver(A_t, b_t, loss=bc.LOSS_LOGISTIC, precision=bc.PREC_FP32, N=wl["N"], M=wl["M"],
                   kappa=wl["kappa"], gamma=wl["gamma"], rho_c=wl["rho"],
                   stream=torch.cuda.current_stream()) as s:
        s.step(1)
        st1 = s.state()
        s.step(1)
        st2 = s.state()
        cons = [consensus_state(s)]          # iteration 2
        for _ in range(6):                   # iterations 3..8
            s.step(1)
            cons.append(consensus_state(s))
    r0, r1 = synth.split_ranges(wl["m"], wl["N"])[0]
    A0 = A[r0:r1].astype(np.float64)
    return wl, b, A0, st1, st2, (r0, r1), cons


def test_iteration1_omega_every_row(run):
    wl, b, A0, st1, st2, _, _cons = run
    want = ref.omega_prox(ref.LOSS_LOGISTIC, np.zeros_like(b), b, wl["M"], wl["rho"])
    assert np.max(np.abs(st1["omega"] - want)) <= TOL32 * np.max(np.abs(want))
    np.testing.assert_allclose(st1["nu"], -st1["omega"], rtol=0, atol=TOL32 * np.max(np.abs(want)))
    assert np.all(st1["x"] == 0) and np.all(st1["z"] == 0) and np.all(st1["u"] == 0)


def test_iteration2_shard0_against_oracle(run):
    wl, b, A0, st1, st2, (r0, r1), _cons = run
    o = ref.BiCADMM(A0, b[r0:r1], ref.LOSS_LOGISTIC, 1, wl["M"], wl["kappa"], gamma=wl["gamma"],
                    rho_c=wl["rho"], n_shards_total=wl["N"])
    o.x_step_shard(0)          # iteration 1 (z = u = 0)
    o.x_step_shard(0)          # iteration 2 (z = u = 0 after iteration 1)
    x0 = st2["x"][0]
    assert np.max(np.abs(x0 - o.x[0])) <= TOL32 * np.max(np.abs(o.x[0]))
    assert np.max(np.abs(st2["omega"][r0:r1] - o.omega)) <= TOL32 * np.max(np.abs(o.omega))
    assert np.max(np.abs(st2["nu"][r0:r1] - o.nu)) <= TOL32 * np.max(np.abs(o.nu))


def test_iteration2_consensus_properties(run):
    wl, b, A0, st1, st2, _, _cons = run
    z, s, x, u = st2["z"], st2["s"], st2["x"], st2["u"]
    kappa = wl["kappa"]
    # u after iteration 2 = u1 + x2 - z2 with u1 = 0
    np.testing.assert_allclose(u, x - z[None, :], rtol=0, atol=1e-12 * max(1.0, np.abs(x).max()))
    # s: at most kappa nonzeros, on the top-kappa |z| (ties lowest index), all of one magnitude
    nz = np.flatnonzero(s)
    assert len(nz) <= kappa
    if len(nz):
        assert set(nz) <= set(ref.top_kappa(z, kappa))
        mags = np.abs(s[nz])
        assert np.all(mags <= 1 + 1e-15) and np.ptp(mags) <= 1e-12
        assert np.all(np.sign(s[nz]) == np.sign(z[nz]))
    # (z, t) with w = mean_i(x_i + u1_i) = mean_i x_i: z = S_tau(w + tau s_prev) and
    # t = ||z||_1 when tau > 0, else z = w; s_prev = s after iteration 1 (= 0 here)
    w = x.mean(axis=0)
    t, tau = st2["t"], st2["tau"]
    s1 = st1["s"]
    y = w + tau * s1
    zz = np.sign(y) * np.maximum(np.abs(y) - tau, 0.0) if tau > 0 else w
    np.testing.assert_allclose(z, zz, rtol=0, atol=1e-9 * max(1.0, np.abs(w).max()))
    if tau > 0:
        assert abs(t - np.abs(z).sum()) <= 1e-9 * max(1.0, t)


def test_consensus_against_oracle_iterations_3_to_8(run):
    """The global step at full size, element by element against the oracle's (z,t) and s
    steps fed with the GPU's own w, s^k and v^k (eqs. global-z-t-updae, s-update-final,
    v-update), from iteration 3 on, where s^k != 0 and the breakpoints of h are nontrivial."""
    wl, *_, cons = run
    taus = []
    for k in range(1, len(cons)):
        assert np.any(cons[k - 1]["s"] != 0), "s^k must be nonzero from iteration 2 on"
        taus.append(check_consensus_step(cons[k - 1], cons[k], wl["N"], wl["rho"], 0.5 * wl["rho"],
                                         wl["kappa"]))
    assert max(taus) > 0.0, "the l1 constraint was never active"
