"""Device memory through the caller's allocator (polar_mesh_desc.alloc / free): every
device buffer of a context -- the multigrid levels, the Krylov vectors, the source fields
allocated by polar_set_coeffs and the schedule arrays grown by polar_advance -- comes from
the hook, and polar_mesh_destroy hands every one back."""
import numpy as np
import pytest

import polar_inputs as pi
from oracle import polar_oracle as po

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2509_15879_gb300")
from paper_2509_15879_gb300 import driver  # noqa: E402


class CountingAllocator(P.TorchAllocator):
    """PyTorch's caching allocator with a ledger of live blocks."""

    def __init__(self):
        self.live, self.allocs, self.frees, self.bytes = {}, 0, 0, 0

    def alloc(self, nbytes, stream):
        p = super().alloc(nbytes, stream)
        self.live[p] = nbytes
        self.allocs += 1
        self.bytes += nbytes
        return p

    def free(self, ptr, stream):
        assert ptr in self.live, "freed a pointer the allocator never handed out"
        del self.live[ptr]
        self.frees += 1
        super().free(ptr, stream)


@pytest.mark.parametrize("precision", [P.POLAR_FP64, P.POLAR_MIXED])
def test_every_buffer_goes_through_the_hooks(precision):
    prob = pi.continuity_problem(40, 72, 6, 21, pe_target=6.0, d_amp=1.3, delta=0.2)
    alloc = CountingAllocator()
    before = torch.cuda.memory_allocated()
    ctx = driver.create(prob, precision, allocator=alloc)
    created = alloc.allocs
    # 7 levels for m = 40, each with a dozen or more arrays, plus the solver vectors
    assert created > 80, created
    assert torch.cuda.memory_allocated() - before >= alloc.bytes
    driver.advance(ctx, prob, 0, 1)
    driver.advance(ctx, prob, 1, 6)           # a longer schedule grows its device arrays
    assert alloc.allocs > created
    U, _ = P.polar_get_state(ctx)
    ref = po.run(prob, 6)
    tol = 1e-12 if precision == P.POLAR_FP64 else 1e-9
    err = float(np.max(np.abs(U - ref)) / np.max(np.abs(ref)))
    print(f"hooked allocator, precision {precision}: {alloc.allocs} allocations, "
          f"{alloc.bytes / 1e6:.1f} MB, rel err vs oracle {err:.2e}")
    assert err < tol
    P.polar_mesh_destroy(ctx)
    assert alloc.frees == alloc.allocs and not alloc.live


def test_allocator_failure_is_reported_and_cleaned_up():
    """An allocator that runs dry part-way through polar_mesh_create: POLAR_ENOMEM, and
    every block handed out before is given back."""

    class Dry(CountingAllocator):
        def alloc(self, nbytes, stream):
            if self.allocs >= 25:
                return 0
            return super().alloc(nbytes, stream)

    prob = pi.continuity_problem(20, 32, 2, 5, pe_target=4.0, delta=0.2)
    alloc = Dry()
    with pytest.raises(P.PolarError) as e:
        P.polar_mesh_create(prob.r, prob.theta, prob.scheme, P.POLAR_FP64, None, alloc)
    assert e.value.code == P.POLAR_ENOMEM
    assert alloc.allocs == 25 and alloc.frees == 25 and not alloc.live
