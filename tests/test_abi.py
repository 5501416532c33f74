"""The C-ABI library loads and exports every entry point include/vmc.h declares; the
ctypes structs of the binding have the C layout; argument validation needs no GPU."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2108_03409_b300 import build as vbuild
from paper_2108_03409_b300 import vmc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vmc.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vmc_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    vbuild.build()
    return vmc.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(vmc.EXPORTED) | set(names)
    assert set(vmc.EXPORTED) == set(names)


def test_struct_layout_matches_header():
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "vmc.h"
#define F(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("vmc_lattice %zu\nvmc_config %zu\nvmc_sr_stats %zu\n", sizeof(vmc_lattice),
         sizeof(vmc_config), sizeof(vmc_sr_stats));
  printf("vmc_tdvp_opts %zu\nvmc_tdvp_stats %zu\n", sizeof(vmc_tdvp_opts), sizeof(vmc_tdvp_stats));
  printf("vmc_excited_stats %zu\n", sizeof(vmc_excited_stats));
  F(vmc_excited_stats, ess) F(vmc_excited_stats, tdvp) F(vmc_sr_stats, solver_relres_explicit)
  F(vmc_lattice, J) F(vmc_lattice, alpha) F(vmc_config, shift) F(vmc_config, cg_tol)
  F(vmc_config, solver) F(vmc_config, tdvp) F(vmc_config, ar_ansatz) F(vmc_config, cnn_ansatz) F(vmc_sr_stats, n_samples)
  F(vmc_sr_stats, solver_relres) F(vmc_sr_stats, ms_update) F(vmc_sr_stats, solver_converged)
  F(vmc_tdvp_opts, eps_snr) F(vmc_tdvp_opts, exact) F(vmc_tdvp_opts, jacobi_max_sweeps)
  F(vmc_tdvp_stats, kept) F(vmc_tdvp_stats, jacobi_off) F(vmc_tdvp_stats, ms)
  F(vmc_tdvp_stats, ms_eig)
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split("\n")
    got = dict(l.rsplit(" ", 1) for l in out if l.strip())
    assert int(got["vmc_lattice"]) == ctypes.sizeof(vmc.vmc_lattice)
    assert int(got["vmc_config"]) == ctypes.sizeof(vmc.vmc_config)
    assert int(got["vmc_sr_stats"]) == ctypes.sizeof(vmc.vmc_sr_stats)
    assert int(got["vmc_tdvp_opts"]) == ctypes.sizeof(vmc.vmc_tdvp_opts)
    assert int(got["vmc_tdvp_stats"]) == ctypes.sizeof(vmc.vmc_tdvp_stats)
    assert int(got["vmc_excited_stats"]) == ctypes.sizeof(vmc.vmc_excited_stats)
    for key, val in got.items():
        if "." in key:
            t, f = key.split(".")
            assert getattr(getattr(vmc, t), f).offset == int(val), key


@pytest.mark.parametrize("bad", [
    dict(n_chains=0), dict(samples_per_chain=0), dict(sweeps_per_sample=0), dict(solver=7),
    dict(precision=5), dict(shift=-1.0), dict(shift_mode=3), dict(tdvp=2),
    dict(ar_ansatz=1), dict(ar_ansatz=1, made_hidden=32, solver=1), dict(cnn_ansatz=1),
])
def test_init_rejects_bad_config_without_gpu(lib, bad):
    cfg = vmc.make_config(**bad)
    lat = vmc.make_lattice(vmc.MODEL_TFIM, 10, 1, 1.0, 1.0, 1)
    with pytest.raises(vmc.VmcError) as e:
        vmc.vmc_init(cfg, [lat])
    assert e.value.status == vmc.VMC_ERR_ARG


@pytest.mark.parametrize("lat", [
    dict(model=2, Lx=4), dict(model=0, Lx=1, Ly=1), dict(model=0, Lx=64, Ly=64),
    dict(model=1, Lx=16, Ly=16, alpha=3), dict(model=0, Lx=4, alpha=0),
])
def test_init_rejects_bad_lattice_without_gpu(lib, lat):
    cfg = vmc.make_config()
    L = vmc.make_lattice(lat.get("model", 0), lat.get("Lx", 4), lat.get("Ly", 1), 1.0, 1.0,
                         lat.get("alpha", 1))
    with pytest.raises(vmc.VmcError) as e:
        vmc.vmc_init(cfg, [L])
    assert e.value.status == vmc.VMC_ERR_ARG


def test_null_context_is_rejected(lib):
    assert lib.vmc_logpsi(None, 0, None, 0, None) == vmc.VMC_ERR_ARG
    assert lib.vmc_sr_step(None, 0, 0.1, None) == vmc.VMC_ERR_ARG
    assert lib.vmc_tdvp_rhs(None, 0, None, 0, None, None, None, None) == vmc.VMC_ERR_ARG
    assert lib.vmc_tdvp_step(None, 0, None, None, None, None) == vmc.VMC_ERR_ARG
    assert lib.vmc_excited_step(None, 0, 1, 0.1, None, None) == vmc.VMC_ERR_ARG
    assert lib.vmc_kernel_launches(None) == 0
    lib.vmc_destroy(None)
