"""roam_bucket_static, the allocation-free bucketing entry point, against the
context-based roam_bucket.  Collected last (file name) so that a stop-at-
first-failure run has already run every other test.

roam_bucket_static serves callers that may not allocate device memory (a
host whose pool allocator owns all device memory, or a frame loop that cannot
take the synchronisation cudaFree implies): it keeps its scratch in a fixed
device array, so these tests also check that the array's leftovers from the
previous call do not leak into the next one."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def roam():
    import paper_2208_02705_gb300 as roam
    from paper_2208_02705_gb300 import build
    build.build()
    return roam


def _ctx_with_fields(roam, n_fields):
    """A context whose field count is n_fields (fully occupied 32^3 grid)."""
    import fixtures as F
    r = roam.Roam(0)
    occ = np.ones((32, 32, 32), dtype=bool)
    r.load_grid(F.pack_bits(occ), (32, 32, 32), (0, 0, 0), 0.1)
    labels = (np.arange(occ.size) % n_fields).astype(np.uint16)
    aff = np.tile(np.array([1, 1, 1, 0, 0, 0], np.float32), (n_fields, 1))
    r.load_fields(labels, aff)
    return r


def _static_bucket(roam, keys_t, n_fields):
    """Calls the C entry point directly with caller-owned buffers."""
    L = roam.load_library()
    n = int(keys_t.shape[0])
    perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    offsets = torch.full((n_fields + 1,), -1, dtype=torch.int32, device="cuda")
    st = L.roam_bucket_static(keys_t.data_ptr() if n else None, n, n_fields, perm.data_ptr(), offsets.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    assert st == 0, L.roam_last_error().decode()
    return perm[:n], offsets


def _same_grouping(keys, perm_a, off_a, perm_b, off_b, n_fields):
    """Offsets are unique and must match exactly; within a field the order is
    unspecified, so compare each field's set of sample indices."""
    assert np.array_equal(off_a, off_b)
    assert np.array_equal(off_a, np.concatenate([[0], np.cumsum(np.bincount(keys, minlength=n_fields))]))
    for f in range(n_fields):
        sa = np.sort(perm_a[off_a[f]:off_a[f + 1]])
        sb = np.sort(perm_b[off_b[f]:off_b[f + 1]])
        assert np.array_equal(sa, sb)
        assert (keys[sa] == f).all()


def test_static_bucket_matches_context_bucket_on_two_calls_in_a_row(roam):
    n_fields = 512
    r = _ctx_with_fields(roam, n_fields)
    rng = np.random.default_rng(2024)
    # two different key sets back to back: the second call must not see the
    # first call's histogram, cursors or counters
    batches = [np.minimum(rng.zipf(1.2, 200003) - 1, n_fields - 1), rng.integers(0, n_fields, 77777)]
    for keys in batches:
        keys_t = torch.from_numpy(keys.astype(np.int16)).cuda()
        perm_s, off_s = _static_bucket(roam, keys_t, n_fields)
        perm_c, off_c = r.bucket(keys_t)
        torch.cuda.synchronize()
        _same_grouping(keys, perm_s.cpu().numpy().astype(np.int64), off_s.cpu().numpy().astype(np.int64),
                       perm_c.cpu().numpy().astype(np.int64), off_c.cpu().numpy().astype(np.int64), n_fields)
    r.check()
    r.close()


def test_static_bucket_limits_and_edges(roam):
    L = roam.load_library()
    keys = torch.zeros(16, dtype=torch.int16, device="cuda")
    perm = torch.empty(16, dtype=torch.int32, device="cuda")
    off = torch.empty(4098, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert L.roam_bucket_static(keys.data_ptr(), 16, 4097, perm.data_ptr(), off.data_ptr(), s) == -1
    assert b"4096" in L.roam_last_error()
    assert L.roam_bucket_static(keys.data_ptr(), 16, 0, perm.data_ptr(), off.data_ptr(), s) == -1
    # empty input: offsets all zero
    p, o = _static_bucket(roam, torch.empty(0, dtype=torch.int16, device="cuda"), 7)
    torch.cuda.synchronize()
    assert (o.cpu().numpy() == 0).all()
    # the largest field count, one sample per field plus a long run in the last field
    n_fields = 4096
    keys = np.concatenate([np.arange(n_fields), np.full(5000, n_fields - 1)])
    p, o = _static_bucket(roam, torch.from_numpy(keys.astype(np.uint16).view(np.int16)).cuda(), n_fields)
    torch.cuda.synchronize()
    o = o.cpu().numpy().astype(np.int64)
    assert o[-1] == keys.size and o[1] == 1 and o[n_fields - 1] == n_fields - 1
    p = p.cpu().numpy().astype(np.int64)
    assert np.array_equal(np.sort(p), np.arange(keys.size))


def test_static_bucket_drops_ids_beyond_n_fields_and_keeps_the_rest(roam):
    """Ids >= n_fields are dropped: offsets[n_fields] counts the kept samples,
    the kept ones are grouped as usual, and perm past the kept count is left
    as it was."""
    n_fields = 100
    rng = np.random.default_rng(7)
    keys = rng.integers(0, 130, 5000)
    perm, off = _static_bucket(roam, torch.from_numpy(keys.astype(np.int16)).cuda(), n_fields)
    torch.cuda.synchronize()
    off = off.cpu().numpy().astype(np.int64)
    perm = perm.cpu().numpy().astype(np.int64)
    kept = keys < n_fields
    assert off[-1] == kept.sum()
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(np.bincount(keys[kept], minlength=n_fields))]))
    assert np.array_equal(np.sort(perm[:off[-1]]), np.nonzero(kept)[0])
    assert (perm[off[-1]:] == -1).all()


def test_static_bucket_allocates_no_device_memory(roam):
    """Repeated calls with caller-owned buffers leave the device's free
    memory exactly as it was (after a first call that looked the scratch
    array up)."""
    n_fields = 300
    keys = torch.from_numpy(np.random.default_rng(9).integers(0, n_fields, 100000).astype(np.int16)).cuda()
    perm = torch.empty(keys.shape[0], dtype=torch.int32, device="cuda")
    off = torch.empty(n_fields + 1, dtype=torch.int32, device="cuda")
    L = roam.load_library()
    s = torch.cuda.current_stream().cuda_stream
    assert L.roam_bucket_static(keys.data_ptr(), keys.shape[0], n_fields, perm.data_ptr(), off.data_ptr(), s) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(20):
        assert L.roam_bucket_static(keys.data_ptr(), keys.shape[0], n_fields, perm.data_ptr(), off.data_ptr(), s) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
