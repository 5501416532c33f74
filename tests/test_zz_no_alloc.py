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
        E = cplx(e)
    assert np.max(np.abs(mog - Oh.mean(axis=0))) <= 1e-6 * max(1.0, np.max(np.abs(mog)))
    if model == T:
        # independently of the CUDA path: the FP64 oracle's F and <O> from the same samples and
        # the same (FP32) local energies, at the stated FP32 reduction bound
        Oref = oracle.ok(N, M, p, s)
        _, Fo, _ = oracle.sr_matrices(Oref, E, want_S=False)
        assert np.max(np.abs(Fg - Fo)) <= F_REL * np.max(np.abs(Fo))
        assert np.max(np.abs(mog - Oref.mean(axis=0))) <= F_REL * max(1.0, np.max(np.abs(mog)))


def test_noalloc_accepts_the_largest_batch_the_scratch_holds():
    """N = 64, M = 128: 62 chunks of 1024 samples fill the array; the call at exactly that
    size is accepted and gives F of the definition (FP64 sums on the host of synthetic
    tanh theta values, spins and energies)."""
    N, M, n = 64, 128, 62 * 1024
    rng = np.random.default_rng(5)
    s = inputs.random_sz0_spins(n, N, seed=6)
    t = (rng.uniform(-0.5, 0.5, (n, M)) + 1j * rng.uniform(-0.5, 0.5, (n, M))).astype(np.complex64)
    E = (rng.normal(-100, 3, n) + 1j * rng.normal(0, 0.1, n)).astype(np.complex64)
    sd = to_dev_spins(s)
    td = torch.from_numpy(np.stack([t.real, t.imag], axis=-1).copy()).cuda()
    ed = torch.from_numpy(np.stack([E.real, E.imag], axis=-1).copy()).cuda()
    P = N + M + N * M
    F = torch.zeros((P, 2), dtype=torch.float64, device="cuda")
    vmc.vmc_force_noalloc(sd, td, ed, N, M, F, None)
    torch.cuda.synchronize()
    Fg = cplx(F)
    Ec = E.astype(np.complex128)
    u = (Ec - Ec.mean()) / n
    sf = s.astype(np.float64)
    tc = t.astype(np.complex128)
    Fa = sf.T @ u
    Fb = tc.conj().T @ u
    Fw = (tc.conj() * u[:, None]).T @ sf                  # [M][N]
    Fref = np.concatenate([Fa, Fb, Fw.reshape(-1)])
    assert np.max(np.abs(Fg - Fref)) <= F_REL * np.max(np.abs(Fref))


def test_noalloc_rejects_sizes_beyond_the_scratch():
    lib = vmc.load()
    x = torch.zeros(16, dtype=torch.int8, device="cuda")
    # N = 64, M = 128: 4 * 129 * 65 doubles per 1024 samples; 2^21 doubles fit 62 chunks
    n_too_big = 63 * 1024
    st = lib.vmc_force_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), n_too_big, 64, 128,
                               x.data_ptr(), None, None)
    assert st == vmc.VMC_ERR_ARG
    assert lib.vmc_force_noalloc(None, None, None, 10, 4, 4, None, None, None) == vmc.VMC_ERR_ARG
    # N = M = 1 fits 2^17 chunks in the array but the grid holds at most 65535
    n_grid = 65536 * 1024
    st = lib.vmc_force_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), n_grid, 1, 1,
                               x.data_ptr(), None, None)
    assert st == vmc.VMC_ERR_ARG
