"""The binding of hcg_preorder_noalloc checks its tensors before calling the
library (no GPU needed): the library writes n values to each output, so a
short, strided, wrongly typed or host-resident tensor must raise instead of
letting a kernel write past the caller's allocation."""
import pytest
import torch

import paper_2012_13173_gb300 as H


def _args(n=8, out_n=None, out_dtype=torch.int64, perm_dtype=torch.int32):
    out_n = n if out_n is None else out_n
    lon = torch.zeros(n, dtype=torch.float64)
    return lon, lon.clone(), torch.zeros(out_n, dtype=out_dtype), torch.zeros(out_n, dtype=perm_dtype)


@pytest.mark.parametrize("case", ["short", "dtype", "perm_dtype", "strided", "host", "lon_2d"])
def test_bad_tensors_raise_before_the_call(case):
    lon, lat, ps, pm = _args()
    if case == "short":
        lon, lat, ps, pm = _args(out_n=7)
    elif case == "dtype":
        lon, lat, ps, pm = _args(out_dtype=torch.int32)
    elif case == "perm_dtype":
        lon, lat, ps, pm = _args(perm_dtype=torch.int64)
    elif case == "strided":
        ps = torch.zeros(16, dtype=torch.int64)[::2]
    elif case == "lon_2d":
        lon = torch.zeros((2, 4), dtype=torch.float64)
    with pytest.raises(H.HcgError, match="INVALID_ARG"):
        H.preorder_noalloc(lon, lat, 16384, 1000, 2000, ps, pm)


def test_check_reports_the_short_tensor():
    lon, lat, ps, pm = _args(n=10, out_n=9)
    with pytest.raises(H.HcgError, match="pix_sorted holds 9 elements"):
        H._check_noalloc_args(lon, lat, ps, pm)
