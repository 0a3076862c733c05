"""The allocation-free mass/momentum entry point (lbm_moments_noalloc).

Callers that cannot allocate device memory when they need these sums (fixed
device budgets, allocators that forbid growth, loops where an allocation
would synchronise the device) use this variant of the FP64 reduction: it
keeps its partial sums in a static device array and only reads the caller's
population array and writes the caller's output.  The test checks its result
against lbm_diagnostics on the same state, on two calls in a row, through the
C ABI.  It is collected last and also passes when run alone.
"""
import ctypes

import numpy as np
import pytest

import lbm_cases as C

pytestmark = pytest.mark.gpu


def _state_populations(solver, case):
    """Device copy of the population block of the solver's state."""
    import torch
    q = 9 if case.lattice == "D2Q9" else 19
    pitch = (case.nx + 7) // 8 * 8
    esz = {"fp32": 4, "fp16": 2, "bf16": 2, "fp64": 8}[case.storage]
    nbytes = q * pitch * case.ny * case.nz * esz
    raw = solver.get_state()[:nbytes].copy()
    return torch.from_numpy(raw).cuda(), q, pitch


# nx = 37 is not a multiple of 8, so rows are padded (pitch 40 > nx); 17,760
# cells take five blocks of the reduction, the last one partial
SIZES = {"D2Q9": (37, 480, 1), "D3Q19": (37, 24, 20)}


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16", "fp64"])
@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q19"])
def test_noalloc_moments_match_diagnostics_twice(lattice, storage):
    import torch
    import paper_2506_03905_gb300 as pkg
    nx, ny, nz = SIZES[lattice]
    # populations stored as f_i - w_i (no reference-velocity shift), the layout
    # the entry point documents
    case = C.channel_3d(re_tau=5200.0, scheme="wall_bb", nx=nx, ny=ny, nz=nz, seed=3,
                        storage=storage).replace(u_shift=0.0, lattice=lattice)
    s = pkg.Solver(case)
    s.set_fields(*C.initial_fields(case))
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for nsteps in (6, 9):              # two calls in a row on changing states
        s.step(nsteps)
        d = s.diagnostics()
        f, q, pitch = _state_populations(s, case)
        assert pitch > nx
        out.fill_(-1.0)
        st = pkg.lbm_moments_noalloc(f.data_ptr(), q, pkg.STORAGE[storage], case.nx, case.ny,
                                     case.nz, pitch, out.data_ptr(), stream)
        assert st == pkg.LBM_OK, pkg.lbm_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = np.array([d.mass, d.momentum[0], d.momentum[1], d.momentum[2]])
        # same FP64 sums in a different partition of the cells
        assert abs(got[0] - ref[0]) <= 1e-12 * abs(ref[0])
        assert np.abs(got[1:] - ref[1:]).max() <= 1e-12 * abs(ref[0])
    s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    import paper_2506_03905_gb300 as pkg
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    st = pkg.lbm_moments_noalloc(dummy.data_ptr(), 19, 0, 4096, 4096, 2, 4096, out.data_ptr(), 0)
    assert st == pkg.LBM_EINVAL
    assert "exceed" in pkg.lbm_last_error(None)
    st = pkg.lbm_moments_noalloc(None, 19, 0, 8, 8, 8, 8, out.data_ptr(), 0)
    assert st == pkg.LBM_EINVAL
