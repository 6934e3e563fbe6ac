"""tsf_zero_pairs_static: the entry point for callers that cannot allocate
device memory (for instance inside a framework that owns all device memory,
or a loop that cannot afford cudaMalloc's implicit synchronisation).  Its
output must equal tsf_zero_pairs's on the same values, call after call, even
though every call reuses one fixed device array left over from the last one.
Collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_no_alloc_zero_pairs_match_the_allocating_entry_point():
    import torch

    import paper_2407_12399_gb300 as tsf
    from paper_2407_12399_gb300 import build as B
    from paper_2407_12399_gb300 import synthetic as S

    B.build()
    cases = [((20, 18, 16), "uniform", 11), ((9, 23, 14), "ties", 12), ((20, 18, 16), "uniform", 11)]
    for shape, kind, seed in cases:  # consecutive calls share the array
        f = S.random_field(shape, seed=seed, kind=kind)
        fld = tsf.Field(torch.from_numpy(f).cuda())
        ref = set(map(tuple, fld.zero_pairs().tolist()))
        fld.close()
        lz, ly, lx = shape
        dev = torch.from_numpy(f).cuda()
        out = torch.zeros(2 * len(ref), dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        r, n = tsf.tsf_zero_pairs_static(lx, ly, lz, dev.data_ptr(), out.data_ptr(), len(ref))
        assert r == tsf.TSF_OK, tsf.tsf_status_string(r)
        assert n == len(ref)
        got = out.cpu().numpy().view(np.uint64).reshape(-1, 2)
        assert set(map(tuple, got.tolist())) == ref


def test_no_alloc_rejects_sizes_beyond_its_array():
    import torch

    import paper_2407_12399_gb300 as tsf
    big = torch.zeros(70 * 70 * 70, dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    r, n = tsf.tsf_zero_pairs_static(70, 70, 70, big.data_ptr(), out.data_ptr(), 1)
    assert r == tsf.TSF_EINVAL


def test_no_alloc_capacity_and_nan_contracts():
    """cap 0 with no output buffer and a cap below the count both report the
    true count with TSF_ECAPACITY; a NaN value is TSF_ENAN."""
    import torch

    import paper_2407_12399_gb300 as tsf
    from paper_2407_12399_gb300 import synthetic as S

    shape = (16, 12, 10)
    f = S.random_field(shape, seed=5, kind="uniform")
    fld = tsf.Field(torch.from_numpy(f).cuda())
    n_true = len(fld.zero_pairs())
    fld.close()
    lz, ly, lx = shape
    dev = torch.from_numpy(f).cuda()
    r, n = tsf.tsf_zero_pairs_static(lx, ly, lz, dev.data_ptr(), None, 0)
    assert r == tsf.TSF_ECAPACITY and n == n_true
    small = torch.zeros(2 * 7, dtype=torch.int64, device="cuda")
    r, n = tsf.tsf_zero_pairs_static(lx, ly, lz, dev.data_ptr(), small.data_ptr(), 7)
    assert r == tsf.TSF_ECAPACITY and n == n_true
    bad = f.copy()
    bad.flat[123] = np.nan
    devb = torch.from_numpy(bad).cuda()
    out = torch.zeros(2 * n_true, dtype=torch.int64, device="cuda")
    r, _ = tsf.tsf_zero_pairs_static(lx, ly, lz, devb.data_ptr(), out.data_ptr(), n_true)
    assert r == tsf.TSF_ENAN
    # and the array still serves a good call afterwards
    r, n = tsf.tsf_zero_pairs_static(lx, ly, lz, dev.data_ptr(), out.data_ptr(), n_true)
    assert r == tsf.TSF_OK and n == n_true
