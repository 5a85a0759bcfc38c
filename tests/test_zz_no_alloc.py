"""The allocation-free distance-graph entry point against the regular graph builder.

sedacs_graph_build_noalloc is for callers that cannot allocate device memory when they call
in (foreign allocators, loops that cannot take cudaMalloc's synchronisation); its scratch is a
fixed array inside the library.  Two calls in a row must both reproduce, bit for bit, the CSR
that sedacs_graph_build writes for the same positions (integer output: bit-exact is the
tolerance), so the shared scratch is reused correctly between calls; a warm call must leave
both the caching allocator's count and the driver's free device memory unchanged.
"""
import numpy as np
import pytest

from paper_2606_03140_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _reference_csr(S, s):
    ctx = S.sedacs_create(s.species, s.box, I.default_model(), S.sedacs_default_params(core_size=12))
    try:
        nnz = S.sedacs_graph_build(ctx, np.ascontiguousarray(s.R))
        return S.sedacs_graph_get(ctx, s.n_atoms, nnz)
    finally:
        S.sedacs_destroy(ctx)


@pytest.mark.parametrize("which", ["water96", "water3000"])
def test_noalloc_graph_matches_regular_builder_twice(which):
    import torch

    from paper_2606_03140_gb300 import sedacs as S

    s = I.workload("water96") if which == "water96" else I.small_water_box(1000, 31.0, seed=33)
    rp_ref, col_ref = _reference_csr(S, s)
    R = torch.from_numpy(np.ascontiguousarray(s.R)).cuda()
    row_ptr = torch.zeros(s.n_atoms + 1, dtype=torch.int64, device="cuda")
    col = torch.full((len(col_ref) + 64,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        row_ptr.zero_()
        col.fill_(-1)
        st, nnz = S.sedacs_graph_build_noalloc(R, s.box, 3.0, row_ptr, col, stream)
        torch.cuda.synchronize()
        assert st == 0 and nnz == len(col_ref)
        assert np.array_equal(row_ptr.cpu().numpy(), rp_ref)
        assert np.array_equal(col[:nnz].cpu().numpy(), col_ref)
    # the call allocates nothing: a warm third call moves neither figure
    torch.cuda.synchronize()
    alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    st, nnz = S.sedacs_graph_build_noalloc(R, s.box, 3.0, row_ptr, col, stream)
    torch.cuda.synchronize()
    alloc1, free1 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    assert st == 0 and nnz == len(col_ref)
    assert alloc1 == alloc0 and free1 == free0, (alloc0, alloc1, free0, free1)


def test_noalloc_rejects_small_output_and_oversized_input():
    import torch

    from paper_2606_03140_gb300 import sedacs as S

    s = I.workload("water96")
    R = torch.from_numpy(np.ascontiguousarray(s.R)).cuda()
    row_ptr = torch.zeros(s.n_atoms + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(10, dtype=torch.int32, device="cuda")
    st, nnz = S.sedacs_graph_build_noalloc(R, s.box, 3.0, row_ptr, col, torch.cuda.current_stream().cuda_stream)
    assert st == 8 and nnz > 10                      # SEDACS_ECAPACITY, size needed reported
    big = torch.zeros((16385, 3), dtype=torch.float64, device="cuda")
    rp_big = torch.zeros(16386, dtype=torch.int64, device="cuda")
    with pytest.raises(S.SedacsError):
        S.sedacs_graph_build_noalloc(big, s.box, 3.0, rp_big, col)
