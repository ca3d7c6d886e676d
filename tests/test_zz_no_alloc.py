"""The allocation-free UC dynamic program (ucac_ucdp_noalloc) against the
workspace variant (ucac_ucdp), through the C ABI.

ucac_ucdp_noalloc exists for callers that may not allocate device memory on
the call path and cannot pass a workspace; its scratch is one static device
array shared by every call.  Two calls in a row (the second smaller, so that
it runs over the first call's leftovers) must give the same decisions and
costs, bit for bit, as ucac_ucdp.  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(rng, T, ng):
    return dict(tau_on=rng.uniform(-0.5, 1.5, (T, ng)), tau_su=rng.uniform(-0.5, 1.5, (T, ng)),
                tau_sd=rng.uniform(-0.5, 1.5, (T, ng)), c0=rng.uniform(0, 3000, ng), csu=rng.uniform(0, 5000, ng),
                csd=rng.uniform(0, 1000, ng), TU=rng.integers(1, 6, ng).astype(np.int32),
                TD=rng.integers(1, 6, ng).astype(np.int32), u0=rng.integers(0, 2, ng).astype(np.int32),
                K0=rng.integers(0, 3, ng).astype(np.int32))


def test_noalloc_matches_workspace_variant_two_calls(ucac_mod):
    import torch
    ucac = ucac_mod
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(2024)
    stream = torch.cuda.current_stream().cuda_stream
    for T, ng in ((48, 6000), (24, 700)):
        x = _inputs(rng, T, ng)
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
        i = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.int32, device=dev)
        A = [f(x["tau_on"]), f(x["tau_su"]), f(x["tau_sd"]), f(x["c0"]), f(x["csu"]), f(x["csd"]), i(x["TU"]),
             i(x["TD"]), i(x["u0"]), i(x["K0"])]
        ptrs = [a.data_ptr() for a in A]
        u_ref = torch.zeros((T, ng), dtype=torch.int8, device=dev)
        c_ref = torch.zeros(ng, dtype=torch.float64, device=dev)
        nbytes = ucac.ucac_ucdp_workspace_bytes(ng, T)
        ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        ucac.ucac_ucdp(ng, T, 1e4, *ptrs, u_ref.data_ptr(), c_ref.data_ptr(), ws.data_ptr(), nbytes, stream)
        u_na = torch.full((T, ng), 7, dtype=torch.int8, device=dev)
        c_na = torch.full((ng,), -1.0, dtype=torch.float64, device=dev)
        ucac.ucac_ucdp_noalloc(ng, T, 1e4, *ptrs, u_na.data_ptr(), c_na.data_ptr(), stream)
        torch.cuda.synchronize()
        assert torch.equal(u_ref, u_na)
        assert torch.equal(c_ref, c_na)


def test_noalloc_rejects_oversized_request(ucac_mod):
    ucac = ucac_mod
    ng, T = 20000, 168
    assert ucac.ucac_ucdp_workspace_bytes(ng, T) > ucac.UCAC_UCDP_NOALLOC_MAX_BYTES
    with pytest.raises(ucac.UcacError, match="static limit"):
        ucac.ucac_ucdp_noalloc(ng, T, 1e4, *([1] * 12))
