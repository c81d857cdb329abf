"""The no-allocation D_DWF entry point against the allocating one.

eofa_dwf_apply_noalloc exists for callers that cannot call cudaMalloc when
they apply the operator (an application whose GPU memory is all handed to
its own pool allocator, or a latency-critical loop that cannot take
cudaMalloc's device synchronisation).  It must give the same result as
eofa_dwf_apply_dev, call after call, although every call reuses the same
static scratch array, and it must not change the device's free memory: the
scratch array is taken when the context is created, never inside the call.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1611_00298_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eofa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_00298_gb300 import eofa as e
    e.load_library()
    return e


@pytest.mark.parametrize("dims,Ls,alpha,mf", [((4, 4, 4, 4), 8, 2.0, 0.04), ((8, 8, 8, 8), 8, 1.0, 0.3)])
def test_noalloc_matches_dwf_apply_dev_twice(eofa, dims, Ls, alpha, mf):
    import torch
    lat = eofa.Lattice(dims, Ls, bc_t=-1)
    lat.gauge_load(inputs.gauge_field(dims, 0.5, 11))
    for call, dagger in enumerate((False, True, False)):
        psi = torch.from_numpy(inputs.fermion5d(dims, Ls, 20 + call)).cuda()
        ref = torch.empty_like(psi)
        got = torch.full_like(psi, np.nan)
        lat.dwf_apply_dev(psi, ref, alpha, 1.8, mf, dagger=dagger)
        lat.dwf_apply_noalloc_dev(psi, got, alpha, 1.8, mf, dagger=dagger)
        torch.cuda.synchronize()
        rel = (torch.linalg.vector_norm(got - ref) / torch.linalg.vector_norm(ref)).item()
        assert rel < 1e-12, (call, dagger, rel)
    lat.close()


@pytest.mark.parametrize("dagger", [False, True])
def test_noalloc_leaves_free_device_memory_unchanged(eofa, dagger):
    """A fresh context, its kernels already loaded by one allocating apply on
    another context: the driver's free-memory count is the same before and
    after two no-allocation calls."""
    import torch
    dims, Ls = (4, 4, 4, 4), 8
    U = inputs.gauge_field(dims, 0.5, 12)
    warm = eofa.Lattice(dims, Ls)
    warm.gauge_load(U)
    psi = torch.from_numpy(inputs.fermion5d(dims, Ls, 30)).cuda()
    ref = torch.empty_like(psi)
    warm.dwf_apply_dev(psi, ref, 2.0, 1.8, 0.04, dagger=dagger)
    lat = eofa.Lattice(dims, Ls)
    lat.gauge_load(U)
    got = torch.empty_like(psi)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        lat.dwf_apply_noalloc_dev(psi, got, 2.0, 1.8, 0.04, dagger=dagger)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    rel = (torch.linalg.vector_norm(got - ref) / torch.linalg.vector_norm(ref)).item()
    assert rel < 1e-12, rel
    lat.close()
    warm.close()


def test_noalloc_rejects_lattices_beyond_the_static_scratch(eofa):
    import torch
    dims, Ls = (8, 8, 8, 8), 16  # 384 V Ls bytes = 24 MiB > 16 MiB
    lat = eofa.Lattice(dims, Ls)
    lat.gauge_load(inputs.gauge_field(dims, 0.1, 1))
    psi = torch.zeros(lat.shape5, dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(psi)
    with pytest.raises(eofa.EOFAError) as ei:
        lat.dwf_apply_noalloc_dev(psi, out, 2.0, 1.8, 0.1)
    assert ei.value.code == eofa.EINVAL
    assert "too large" in str(ei.value)
    lat.close()
