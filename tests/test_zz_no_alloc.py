"""a2ls_apply_static: the apply for callers that cannot have device memory
allocated for them (an application whose device memory is fully reserved by
its own pool allocator, or a latency-critical loop that must not allocate).
It takes its scratch vectors from a fixed 8 MiB array in the library's static
device memory.  Checked against a2ls_apply on two calls in a row, with the
tolerance the parity tests use; a problem that needs more scratch than the
array holds is rejected with A2LS_ERR_ARG.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from workloads import pde

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    from paper_2201_02250_gb300 import _build
    _build.build()


@pytest.mark.parametrize("variant,pou,precision", [
    ("deflated_ras", "boolean", "fp64"),
    ("deflated_ras", "boolean", "fp32"),
    ("deflated_ras", "multiplicity", "fp64"),   # RAS that combines yloc with the coarse q
    ("additive_asm", "multiplicity", "fp64"),
    ("ras", "boolean", "fp64"),
    ("asm", "boolean", "fp64"),                 # yloc right after q and t, no coarse pieces
])
def test_apply_static_matches_apply(variant, pou, precision):
    from paper_2201_02250_gb300 import a2ls
    prob = pde.tiny_conv_diff(m=40, nb=3, overlap=2, nev=5)
    P, _keep = a2ls.from_scipy(prob.A, prob.part, prob.overlap, prob.nev, variant=variant, pou=pou,
                               precision=precision)
    rng = np.random.Generator(np.random.PCG64(5))
    rs = [torch.as_tensor(rng.uniform(-1, 1, prob.n), device="cuda") for _ in range(2)]
    z_refs = [torch.empty_like(r) for r in rs]
    zs = [torch.full_like(r, float("nan")) for r in rs]
    for r, z_ref in zip(rs, z_refs):
        P.apply(r, z_ref)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for call in range(2):   # the first static call after setup included: no device memory is taken
        P.apply_static(rs[call], zs[call])
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before, call
    for call in range(2):
        a, b = zs[call].cpu().numpy(), z_refs[call].cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b), (call, np.linalg.norm(a - b))
    P.close()


def test_apply_static_rejects_oversized_problem():
    from paper_2201_02250_gb300 import a2ls
    n, parts = 600_000, 600
    A = sp.diags([-np.ones(n - 1), 2.0 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    part = (np.arange(n) * parts // n).astype(np.int32)
    P, _keep = a2ls.from_scipy(A, part, 1, 0, variant="ras", precision="fp32")
    r = torch.ones(n, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    with pytest.raises(a2ls.A2lsError) as e:
        P.apply_static(r, z)
    assert e.value.code == a2ls.A2LS_ERR_ARG and "static scratch" in str(e.value)
    P.apply(r, z)  # the regular apply still works on the same handle
    torch.cuda.synchronize()
    assert torch.isfinite(z).all()
    P.close()
