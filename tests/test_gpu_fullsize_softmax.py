"""Parity at the full size of the sparse softmax workload (500000 x 2000, K = 10 classes, A
stored in BF16, N = 32, M = 4, entrywise kappa = 500, rho = 1) in the launch configuration
bench.py times (BF16 precision, automatic panel choice = the tensor-core pass, J = 1), on
outputs the oracle can compute alone, plus properties that hold at any size.

* After iteration 1, W = 0, so every row's omega is the K-vector prox at 0 (eq. p:GPU;omega
  with the cross-entropy loss) and nu = -omega.
* After iteration 1, z = u = 0, so iteration 2's x-step of shard 0 depends on shard 0 only:
  the oracle runs that shard alone (with the global N in the ridge coefficient) on the
  BF16-rounded rows and is compared with x_0, omega and nu of shard 0.
* z, s, t after iteration 2: the s-step / (z,t) relations over the n K flattened entries.
"""
import numpy as np
import pytest

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import bicadmm as bc
from paper_2405_16267_b300 import synth

from gpu_util import check_consensus_step, consensus_state

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def run():
    import torch
    import bench
    wl = dict(bench.SOFTMAX)
    A, b = bench.generate_softmax(wl)
    A_t = torch.from_numpy(A).cuda().to(torch.bfloat16)
    b_t = torch.from_numpy(b).cuda()
    with bc.Solver(A_t, b_t, loss=bc.LOSS_SOFTMAX, precision=bc.PREC_BF16, N=wl["N"], M=wl["M"],
                   K=wl["K"], kappa=wl["kappa"], gamma=wl["gamma"], rho_c=wl["rho"], pass_rows=0,
                   stream=torch.cuda.current_stream()) as s:
        s.step(1)
        st1 = s.state()
        s.step(1)
        st2 = s.state()
        cons = [consensus_state(s)]          # iteration 2
        for _ in range(6):                   # iterations 3..8
            s.step(1)
            cons.append(consensus_state(s))
        lists = bc.get_trace(s.h)["zt_lists"]
    del A_t
    r0, r1 = synth.split_ranges(wl["m"], wl["N"])[0]
    A0 = synth.round_to_bf16(A[r0:r1]).astype(np.float64)
    cons[0]["lists"] = lists
    return wl, b, A0, st1, st2, (r0, r1), cons


def test_iteration1_omega_every_row(run):
    wl, b, A0, st1, st2, _, _cons = run
    want = ref.softmax_prox(np.zeros((len(b), wl["K"])), b.astype(np.int64), wl["M"], wl["rho"])
    scale = np.max(np.abs(want))
    assert np.max(np.abs(st1["omega"] - want)) <= TOL * scale
    np.testing.assert_allclose(st1["nu"], -st1["omega"], rtol=0, atol=TOL * scale)
    assert np.all(st1["x"] == 0) and np.all(st1["z"] == 0) and np.all(st1["u"] == 0)


def test_iteration2_shard0_against_oracle(run):
    wl, b, A0, st1, st2, (r0, r1), _cons = run
    o = ref.BiCADMM(A0, b[r0:r1], ref.LOSS_SOFTMAX, 1, wl["M"], wl["kappa"], gamma=wl["gamma"],
                    rho_c=wl["rho"], n_shards_total=wl["N"], K=wl["K"])
    o.x_step_shard(0)          # iteration 1 (z = u = 0)
    o.x_step_shard(0)          # iteration 2 (z = u = 0 after iteration 1)
    x0 = st2["x"][0]
    assert np.max(np.abs(x0 - o.x[0])) <= TOL * np.max(np.abs(o.x[0]))
    om = np.asarray(o.omega).reshape(r1 - r0, wl["K"])
    nu = np.asarray(o.nu).reshape(r1 - r0, wl["K"])
    assert np.max(np.abs(st2["omega"][r0:r1] - om)) <= TOL * np.max(np.abs(om))
    assert np.max(np.abs(st2["nu"][r0:r1] - nu)) <= TOL * np.max(np.abs(nu))


def test_iteration2_consensus_properties(run):
    wl, b, A0, st1, st2, _, _cons = run
    z, s, x, u = st2["z"], st2["s"], st2["x"], st2["u"]
    kappa = wl["kappa"]
    assert z.shape == (wl["n"] * wl["K"],)
    np.testing.assert_allclose(u, x - z[None, :], rtol=0, atol=1e-12 * max(1.0, np.abs(x).max()))
    nz = np.flatnonzero(s)
    assert len(nz) <= kappa
    if len(nz):
        assert set(nz) <= set(ref.top_kappa(z, kappa))
        mags = np.abs(s[nz])
        assert np.all(mags <= 1 + 1e-15) and np.ptp(mags) <= 1e-12
        assert np.all(np.sign(s[nz]) == np.sign(z[nz]))
    w = x.mean(axis=0)
    t, tau = st2["t"], st2["tau"]
    y = w + tau * st1["s"]
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


def test_consensus_steps_3_to_8_ran_on_the_entry_lists(run):
    """The checked steps are the warm-started list form (only the entries with a breakpoint
    above the previous root or a nonzero z or s are visited) whenever the previous root is
    positive and h stays non-positive there."""
    *_, cons = run
    lists = cons[0]["lists"]
    taus = [c["tau"] for c in cons]
    assert lists.size == len(cons) + 1  # iterations 1..8; cons starts at 2
    assert lists[0] == 0  # iteration 1: tau_prev = 0
    # cons[k] holds the state after iteration k + 2, whose record is lists[k + 1]
    warm = [k for k in range(1, len(cons)) if taus[k - 1] > 0.0]
    assert warm and sum(lists[k + 1] for k in warm) >= 0.5 * len(warm), (lists, taus)
