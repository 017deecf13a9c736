"""sncc_integral_noalloc, the entry point for callers that cannot allocate
device memory where they call the library (a host application that owns the
whole memory budget, a latency-critical loop that cannot take the device-wide
synchronisation of cudaMalloc, or plain C code with no allocator for a
workspace).  It must give exactly the sum tables sncc_integral gives, call
after call, although every call reuses the same built-in scratch array.

This file is collected last on purpose; it also passes when run alone."""
import numpy as np
import pytest

from paper_2502_01286_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sncc():
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA GPU")
    from paper_2502_01286_gb300 import build
    build.build()
    from paper_2502_01286_gb300 import sncc as mod
    return mod


def _reference(sncc, fd, bits):
    tb = sncc.integral(fd, s_bits=bits)
    torch.cuda.synchronize()
    return tb.s.clone(), tb.s2.clone()


@pytest.mark.parametrize("M,N,bits", [(1920, 1080, 32), (4096, 4096, 64)])
def test_noalloc_matches_workspace_entry_point_twice(sncc, M, N, bits):
    """Two calls in a row through the C ABI, on two different sources: each
    result equals sncc_integral's exactly (integer tables, so the test's
    tolerance for them is zero)."""
    first = synth.random_image(31 + M, M, N)
    second = synth.random_image(32 + M, M, N, lo=100)
    for img in (first, second):
        fd = torch.as_tensor(img).cuda()
        ref_s, ref_s2 = _reference(sncc, fd, bits)
        tb = sncc.alloc_tables(M, N, bits)
        tb.s.fill_(-1)
        tb.s2.fill_(-1)
        sncc.integral_noalloc(fd, tb)
        torch.cuda.synchronize()
        assert torch.equal(tb.s[:, :M + 1], ref_s[:, :M + 1])
        assert torch.equal(tb.s2[:, :M + 1], ref_s2[:, :M + 1])


def test_noalloc_shrinking_sizes_leave_no_stale_state(sncc):
    """A large call followed by a small one: the small one must not see what
    the large one left in the shared scratch."""
    big = torch.as_tensor(synth.random_image(7, 3000, 2000)).cuda()
    sncc.integral_noalloc(big)
    small_img = synth.random_image(8, 257, 129)
    fd = torch.as_tensor(small_img).cuda()
    tb = sncc.integral_noalloc(fd, s_bits=32)
    torch.cuda.synchronize()
    ref_s, ref_s2 = _reference(sncc, fd, 32)
    assert torch.equal(tb.s[:, :258], ref_s[:, :258])
    assert torch.equal(tb.s2[:, :258], ref_s2[:, :258])
    # and against the definition (column-then-row cumulative sums)
    want = np.zeros((130, 258), np.int64)
    want[1:, 1:] = small_img.astype(np.int64).cumsum(0).cumsum(1)
    np.testing.assert_array_equal(tb.s[:, :258].cpu().numpy(), want)


def test_noalloc_rejects_sources_beyond_the_scratch(sncc):
    """A source whose band sums need more than the built-in 16 MiB is refused
    with SNCC_ERR_CAPACITY before anything is launched or read (the buffers
    passed here are far too small for the size and are never touched)."""
    M, N = 16383, 65535
    assert sncc.lib().sncc_integral_workspace_bytes(M, N) > sncc.NOALLOC_SCRATCH_BYTES
    dummy = torch.zeros(64, dtype=torch.int64, device="cuda")
    rc = sncc.lib().sncc_integral_noalloc(dummy.data_ptr(), M, N, M, dummy.data_ptr(), 64, dummy.data_ptr(),
                                          sncc.sat_pitch(M), None)
    assert rc == sncc.ERR_CAPACITY
