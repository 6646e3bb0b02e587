"""The allocation-free Coulomb entry point against the regular one (GPU).

pb_coulomb_energy_noalloc is for callers that cannot let the library
allocate device memory (applications that own all device memory through
their own pool, or loops that must avoid the synchronisation of
cudaMalloc/cudaFree).  It must agree with pb_coulomb_energy on consecutive
calls with different charge sets, since every call reuses the same static
scratch array, and it must refuse charge counts beyond that array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from gpu_util import ctx, problem
from synth.configs import protein_atoms, sphere_problem

pytestmark = pytest.mark.gpu


def _reference(xyz, q):
    # the regular entry point needs a problem whose surface encloses the charges
    d = sphere_problem(level=1, radius=60.0)
    d["charges"] = {"xyz": xyz, "q": q, "region": 0}
    return problem(d, theta=-1.0, precision="fp64").coulomb_energy()


def test_noalloc_coulomb_matches_regular_entry_point_twice():
    import torch
    from paper_1309_4018_b300 import pbbem
    ctx()
    at = protein_atoms(2000, 2)
    cases = [(at["xyz"], at["q"]), (at["xyz"][:1500] * 1.1, at["q"][:1500] * -0.7)]
    out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    for xyz, q in cases:
        ref = _reference(np.ascontiguousarray(xyz), np.ascontiguousarray(q))
        xt = torch.tensor(np.ascontiguousarray(xyz), dtype=torch.float64, device="cuda:0")
        qt = torch.tensor(np.ascontiguousarray(q), dtype=torch.float64, device="cuda:0")
        rc, msg = pbbem.coulomb_energy_noalloc(0, xt.data_ptr(), qt.data_ptr(), qt.numel(), 4.0, out.data_ptr(),
                                               stream)
        assert rc == pbbem.PB_OK, msg
        torch.cuda.synchronize()
        assert abs(out.item() - ref) <= 1e-12 * abs(ref)


def test_noalloc_coulomb_rejects_oversized_input():
    import torch
    from paper_1309_4018_b300 import pbbem
    ctx()
    buf = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    rc, msg = pbbem.coulomb_energy_noalloc(0, buf.data_ptr(), buf.data_ptr(), 262145, 4.0, buf.data_ptr(), 0)
    assert rc == pbbem.PB_EINVAL and "262144" in msg
