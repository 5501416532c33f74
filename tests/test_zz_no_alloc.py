"""vmc_force_noalloc: the <O>/F reduction for callers that cannot allocate device memory
(its scratch is a fixed file-scope device array).  Its output must match vmc_grad's on
the same inputs, on two consecutive calls (the second finds the first call's partial
sums still in the shared array)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2108_03409_b300 import inputs
from paper_2108_03409_b300 import vmc

from gpu_helpers import F_REL, context, cplx, lattice, to_dev_spins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T, H = inputs.MODEL_TFIM, inputs.MODEL_HEIS


@pytest.mark.parametrize("case", [(T, 6, 6, 3.0, 2, 3000), (H, 8, 8, 0.0, 2, 1024)],
                         ids=["tfim6x6_n3000", "heis8x8_n1024"])
def test_noalloc_force_matches_grad_twice(case):
    model, Lx, Ly, h, alpha, n = case
    N, M = Lx * Ly, alpha * Lx * Ly
    P = N + M + N * M
    p = inputs.rbm_params(N, M, 0.05, seed=17, marshall=(Lx, Ly) if model == H else None)
    s = inputs.initial_spins(model, n, N, seed=18)
    with context(lattice(model, Lx, Ly, 1.0, h, alpha), n_chains=n, solver=vmc.SOLVER_CG) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        sd = to_dev_spins(s)
        e = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
        vmc.vmc_local_energy(ctx, 0, sd, e)
        O = torch.zeros((n, P, 2), dtype=torch.float32, device="cuda")
        F_ref = torch.zeros((P, 2), dtype=torch.float64, device="cuda")
        vmc.vmc_grad(ctx, 0, sd, e, O, F_ref)
        tanh_theta = O[:, N:N + M, :].contiguous()          # O_{b_j} = tanh theta_j
        torch.cuda.synchronize()
        Fr = cplx(F_ref)
        scale = np.max(np.abs(Fr))
        for _ in range(2):
            F = torch.full((P, 2), float("nan"), dtype=torch.float64, device="cuda")
            mo = torch.full((P, 2), float("nan"), dtype=torch.float64, device="cuda")
            vmc.vmc_force_noalloc(sd, tanh_theta, e, N, M, F, mo)
            torch.cuda.synchronize()
            Fg, mog = cplx(F), cplx(mo)
            assert np.all(np.isfinite(Fg)) and np.all(np.isfinite(mog))
            assert np.max(np.abs(Fg - Fr)) <= F_REL * scale
        Oh = cplx(O)
    assert np.max(np.abs(mog - Oh.mean(axis=0))) <= 1e-6 * max(1.0, np.max(np.abs(mog)))


def test_noalloc_rejects_sizes_beyond_the_scratch():
    lib = vmc.load()
    x = torch.zeros(16, dtype=torch.int8, device="cuda")
    # N = 64, M = 128: 4 * 129 * 65 doubles per 1024 samples; 2^21 doubles fit 62 chunks
    n_too_big = 63 * 1024
    st = lib.vmc_force_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), n_too_big, 64, 128,
                               x.data_ptr(), None, None)
    assert st == vmc.VMC_ERR_ARG
    assert lib.vmc_force_noalloc(None, None, None, 10, 4, 4, None, None, None) == vmc.VMC_ERR_ARG
