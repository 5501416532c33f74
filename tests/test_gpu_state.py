"""Checkpoint / resume through the C ABI, and the failure path of the bounded device waits
(a wait that nothing satisfies must give up with VMC_ERR_TIMEOUT; no GPU fault is involved)."""
import numpy as np
import pytest

from paper_2108_03409_b300 import inputs, vmc

from gpu_helpers import cplx

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T = inputs.MODEL_TFIM


def _ctx(C, H, seed=17, L=6):
    cfg = vmc.make_config(seed=seed, n_chains=C, solver=vmc.SOLVER_CHOLESKY_MIXED,
                          precision=vmc.PREC_BF16SPLIT, shift=1e-3, made_hidden=H, made_batch=1024)
    return vmc.vmc_init(cfg, [vmc.make_lattice(T, L, L, 1.0, 3.0, 2)])


def test_resume_continues_identically():
    """A context restored from a checkpoint continues exactly like the original: same SR
    updates, same chains, same learned-proposal rounds (all randomness is counter-based and
    the counters are part of the state)."""
    L, C, H = 6, 512, 32
    N, M = L * L, 2 * L * L
    a = _ctx(C, H)
    b = _ctx(C, H)
    try:
        vmc.vmc_set_params(a, 0, inputs.rbm_params(N, M, 0.05, seed=5))
        vmc.vmc_set_chains(a, 0, inputs.random_spins(C, N, seed=6))
        vmc.vmc_sr_step(a, 0, 0.02)
        train = torch.zeros((4 * C, N), dtype=torch.int8, device="cuda")
        vmc.vmc_sample(a, 0, 0, 4, train)
        vmc.vmc_made_set_params(a, 0, inputs.made_params(N, H, seed=7))
        vmc.vmc_proposal_train(a, 0, train, epochs=2, lr=1e-3)
        vmc.vmc_sample_learned(a, 0, 2)
        state = vmc.vmc_get_state(a)
        vmc.vmc_set_state(b, state)
        out = []
        for ctx in (a, b):
            st = vmc.vmc_sr_step(ctx, 0, 0.02)
            el = torch.zeros((3 * C, 2), dtype=torch.float32, device="cuda")
            acc = vmc.vmc_sample_learned(ctx, 0, 3, None, el)
            vmc.vmc_proposal_train(ctx, 0, train, epochs=1, lr=1e-3)
            out.append((st.e_mean_re, vmc.vmc_get_params(ctx, 0), vmc.vmc_get_chains(ctx, 0, C, N),
                        acc, cplx(el), vmc.vmc_made_get_params(ctx, 0, H * N + H + H * H + H + N * H + N)))
        (ea, pa, ca, aa, ela, ma), (eb, pb, cb, ab, elb, mb) = out
        assert ea == eb and aa == ab
        assert np.array_equal(pa, pb) and np.array_equal(ca, cb)
        assert np.array_equal(ela, elb) and np.array_equal(ma, mb)
    finally:
        vmc.vmc_destroy(a)
        vmc.vmc_destroy(b)


def test_state_of_another_configuration_is_rejected():
    a = _ctx(256, 32)
    b = _ctx(128, 32)              # different chain count
    c = _ctx(256, 32, L=4)         # different lattice
    try:
        state = vmc.vmc_get_state(a)
        p_before = vmc.vmc_get_params(b, 0)
        for ctx in (b, c):
            with pytest.raises(vmc.VmcError) as ei:
                vmc.vmc_set_state(ctx, state)
            assert ei.value.status == vmc.VMC_ERR_ARG
        assert np.array_equal(vmc.vmc_get_params(b, 0), p_before)
        with pytest.raises(vmc.VmcError):
            vmc.vmc_set_state(a, b"not a state" * 4)
    finally:
        for ctx in (a, b, c):
            vmc.vmc_destroy(ctx)


@pytest.mark.parametrize("which", [0, 1, 2], ids=["flag", "mbarrier", "entry"])
def test_bounded_wait_reports_timeout_and_context_survives(which):
    """The bounded waits of the cooperative kernels (flag), of the tensor-core kernels
    (mbarrier) and of the triangular solves (an entry that is never written) give up on a
    condition that never comes true, the call reports VMC_ERR_TIMEOUT, and the context keeps
    working afterwards."""
    N, M = 10, 10
    ctx = vmc.vmc_init(vmc.make_config(n_chains=64, solver=vmc.SOLVER_CG),
                       [vmc.make_lattice(T, N, 1, 1.0, 1.0, 1)])
    try:
        assert vmc.vmc_selftest_wait_timeout(ctx, which) == vmc.VMC_ERR_TIMEOUT
        p = inputs.rbm_params(N, M, 0.1, seed=3)
        vmc.vmc_set_params(ctx, 0, p)
        s = torch.from_numpy(inputs.random_spins(64, N, seed=4)).cuda()
        out = torch.zeros((64, 2), dtype=torch.float32, device="cuda")
        vmc.vmc_logpsi(ctx, 0, s, out)
        assert np.all(np.isfinite(out.cpu().numpy()))
    finally:
        vmc.vmc_destroy(ctx)
