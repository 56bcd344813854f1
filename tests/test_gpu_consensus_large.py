"""The global step at large n, element by element against the oracle, on inputs built to
stress the top-kappa radix select and the (z,t) root (eqs. global-z-t-updae, s-update-final,
v-update of Sec. 3).

The allocation-free entry point takes w, s^k and v^k directly, so the inputs are
constructed rather than reached by iterating.  w holds (all at random positions):
  * a clear top of 3 kappa / 5 entries with |w| in [3, 4);
  * an exact tie group of kappa entries with |w| = 2 and s = 0, so |z| = 2 - tau ties
    exactly and the kappa-th largest |z| falls inside the group: the lowest indices win;
  * 64 entries next to 2 whose bit patterns differ from it by +-1, +-255, +-256, +-257,
    +-65535, +-65536, +-2^24 and +-(2^32 + 1) units in the last place, i.e. across the
    8-bit digit boundaries of the select;
  * small entries |w| < 0.01 elsewhere; s != 0 on half the top and on 2 kappa small
    entries, s = sign(w) exactly on 50 entries (breakpoints at infinity).
v < 0 makes h(0) < 0 (the l1 constraint active) except in the case built to be inactive.
Two calls run back to back (the second on the first call's s and v, with a new w), at
n = 20000 and at the entry point's maximum n = 32768 (= 32 x 1024, a whole number of
32-entry chunks for the 1024-thread CTA).
"""
import numpy as np
import pytest

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import bicadmm as bc

pytestmark = pytest.mark.gpu

TOL = 1e-9


def make_w_s(n, kappa, seed):
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    mags = rng.uniform(0.0, 0.01, n)
    nb = 3 * kappa // 5
    big, tie = perm[:nb], perm[nb:nb + kappa]
    near = perm[nb + kappa:nb + kappa + 64]
    rest = perm[nb + kappa + 64:]
    mags[big] = 3.0 + rng.uniform(0.0, 1.0, nb)
    mags[tie] = 2.0
    offs = np.array([1, -1, 255, -255, 256, -256, 257, -257, 65535, -65535, 65536, -65536,
                     1 << 24, -(1 << 24), (1 << 32) + 1, -(1 << 32) - 1], dtype=np.int64)
    mags[near] = (np.float64(2.0).view(np.int64) + np.resize(offs, near.size)).view(np.float64)
    w = mags * rng.choice([-1.0, 1.0], n)
    s = np.zeros(n)
    on = np.concatenate([big[: nb // 2], rest[: 2 * kappa]])
    s[on] = rng.uniform(-1.0, 1.0, on.size)
    exact = rest[2 * kappa: 2 * kappa + 50]
    s[exact] = np.sign(w[exact])
    return w, s, tie


CASES = [
    # (n, kappa, N, rho_c, rho_b, v0)
    (20000, 500, 64, 10.0, 0.5, -50.0),      # kappa-th |z| inside the tie group
    (32768, 500, 64, 10.0, 0.5, -50.0),      # the same at the maximum n
    (32768, 3000, 64, 10.0, 0.5, -50.0),     # a wider kappa
    (32768, 500, 16, 4.0, 1.0, -5.0),        # ties thresholded to 0: kappa > nnz(z)
    (20000, 20000, 64, 10.0, 0.5, -50.0),    # kappa = n
    (20000, 500, 64, 10.0, 0.5, 1.0e5),      # h(0) >= 0: constraint inactive, z = w
]


@pytest.mark.parametrize("case", CASES)
def test_consensus_large_n_with_ties(case):
    import torch
    n, kappa, N, rho_c, rho_b, v0 = case
    w1, s0, tie = make_w_s(n, kappa, seed=n + kappa)
    rng = np.random.default_rng(7)
    w2 = w1 * (1.0 + 0.01 * rng.standard_normal(n))
    w2[tie] = w1[tie]                   # the tie group stays tied in the second call
    dev = torch.device("cuda")
    z = torch.zeros(n, dtype=torch.float64, device=dev)
    s = torch.tensor(s0, dtype=torch.float64, device=dev)
    tvt = torch.tensor([0.0, v0, 0.0, 0.0], dtype=torch.float64, device=dev)
    v = v0
    s_prev = s0
    for call, w in enumerate((w1, w2)):
        wz, wt, wtau = ref.zt_step(w, s_prev, v, N, rho_c, rho_b)
        bc.consensus_step_noalloc(torch.tensor(w, dtype=torch.float64, device=dev), z, s, tvt, kappa, N, rho_c, rho_b)
        torch.cuda.synchronize()
        zg, sg, tv = z.cpu().numpy(), s.cpu().numpy(), tvt.cpu().numpy()
        assert tv[3] == 0.0, "device status"
        zs = float(np.max(np.abs(wz)))
        assert float(np.max(np.abs(zg - wz))) <= TOL * zs, (call, "z")
        assert abs(tv[0] - wt) <= TOL * max(abs(wt), zs), (call, "t", tv[0], wt)
        assert abs(tv[2] - wtau) <= TOL * max(wtau, 1e-12), (call, "tau", tv[2], wtau)
        if v0 < 0 and call == 0:
            assert wtau > 0.0
        # s from the GPU's own z and t: the same selected entries (lowest-index ties)
        ws = ref.s_step(zg, tv[0], v, kappa)
        assert np.array_equal(sg != 0, ws != 0), (call, "selected entries")
        assert float(np.max(np.abs(sg - ws))) <= 1e-12, (call, "s")
        wv = v + float(zg @ sg) - tv[0]
        assert abs(tv[1] - wv) <= TOL * max(abs(wv), abs(tv[0]), 1e-12), (call, "v")
        if call == 0 and kappa < n and v0 < 0 and N == 64:
            # the constructed tie group straddles the kappa boundary
            sel = set(ref.top_kappa(zg, kappa).tolist())
            assert 0 < len(sel & set(tie.tolist())) < len(tie)
        v, s_prev = tv[1], sg
