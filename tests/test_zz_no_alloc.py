"""sblm_ea_generation_noalloc: the generation of sblm_ea_generation with its scratch in a fixed
device array, for callers that must not allocate device memory while they run. Called here
through the C ABI and compared with sblm_ea_generation on two calls in a row. (This file is
named so that pytest collects it last.)"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
GENE_TOL = 1e-15  # the tolerance of the other EA parity tests


def _chi2(rng, n_pop):
    chi = rng.uniform(0, 100, n_pop)
    chi[rng.choice(n_pop, 3, replace=False)] = np.nan
    chi[5] = chi[7]
    return torch.tensor(chi, device="cuda")


@pytest.mark.parametrize("n_pop,n_par", [(64, 6), (4096, 6), (2048, 16)])
def test_noalloc_matches_generation_twice(lib, n_pop, n_par):
    rng = np.random.default_rng(n_pop + n_par)
    p = lib.params(n_pop=n_pop, seed=21, p_mut0=0.05)
    P_ref = torch.empty((n_pop, n_par), dtype=torch.float64, device="cuda")
    st_ref = lib.new_state_buffer("cuda")
    lib.ea_init(P_ref, n_par, p, 4, st_ref)
    P_new, st_new = P_ref.clone(), st_ref.clone()
    for gen in range(2):
        chi = _chi2(rng, n_pop)
        lib.ea_generation(P_ref, chi, p, 4, gen, st_ref)
        status = lib._lib.sblm_ea_generation_noalloc(
            P_new.data_ptr(), chi.data_ptr(), n_pop, n_par, ctypes.byref(p), 4, gen, st_new.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
        assert status == 0, lib._lib.sblm_last_error()
        torch.cuda.synchronize()
        assert torch.max(torch.abs(P_new - P_ref)).item() <= GENE_TOL
        a, b = lib.read_state(st_ref), lib.read_state(st_new)
        assert (a.p_mut, a.best_chi2, a.n_hist, a.stag_run, a.n_restarts, a.generation) == \
               (b.p_mut, b.best_chi2, b.n_hist, b.stag_run, b.n_restarts, b.generation)


def test_noalloc_rejects_what_it_cannot_hold(lib):
    p = lib.params(n_pop=8192, seed=1)
    P = torch.zeros((8192, 6), dtype=torch.float64, device="cuda")
    chi = torch.zeros(8192, dtype=torch.float64, device="cuda")
    st = lib.new_state_buffer("cuda")
    with pytest.raises(lib.SBLMError, match="fixed scratch"):
        lib.ea_generation_noalloc(P, chi, p, 0, 0, st)
    p = lib.params(n_pop=16, seed=1)
    with pytest.raises(lib.SBLMError, match="device memory only"):
        lib.ea_generation_noalloc(np.zeros((16, 6)), np.zeros(16), p, 0, 0, st)
