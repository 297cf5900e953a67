"""Systematic resampling through the entry point that allocates nothing.

pf_systematic_resample_noalloc serves callers that can neither allocate device
memory nor hand over scratch when they resample (host frameworks that own every
allocation, real-time loops with a fixed memory budget); it uses a device array
built into the library.  Its ancestors must equal those of
pf_systematic_resample (whose scratch the caller allocates) exactly -- this is
index work -- on two calls in a row, since every call reuses the same array.
This file is collected last so that a failure here leaves every other test run.
"""
import numpy as np
import pytest

from paper_1407_8071_gb300 import pf, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _inputs(N, seed):
    kinds = ["lognormal", "spike", "ties", "sparse", "uniform"]
    w = np.concatenate([W.random_weights(int(n), seed=seed + i, kind=kinds[i % len(kinds)])
                        for i, n in enumerate(N)])
    u = W.random_uniforms(len(N), seed=seed)
    return torch.from_numpy(w).cuda(), torch.from_numpy(u).cuda()


def _with_caller_scratch(N, d_w, d_u, stream=None):
    d_anc = torch.empty(d_w.numel(), dtype=torch.int32, device="cuda")
    d_scr = torch.empty(pf.pf_systematic_scratch_bytes(len(N), d_w.numel()), dtype=torch.uint8, device="cuda")
    pf.pf_systematic_resample(N, d_w, d_u, d_anc, d_scr, stream=stream)
    torch.cuda.synchronize()
    return d_anc.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice():
    calls = [
        np.array([1, 7, 1023, 1024, 1025, 4096, 300], dtype=np.int32),
        W.ragged_counts(40, 64, 4096),  # a second, different problem reusing the same array
    ]
    for k, N in enumerate(calls):
        d_w, d_u = _inputs(N, seed=100 + k)
        d_anc = torch.full((d_w.numel(),), -7, dtype=torch.int32, device="cuda")
        pf.pf_systematic_resample_noalloc(N, d_w, d_u, d_anc)
        torch.cuda.synchronize()
        got = d_anc.cpu().numpy()
        assert np.array_equal(got, _with_caller_scratch(N, d_w, d_u)), k


def test_noalloc_on_a_stream_of_the_callers():
    """Callers normally pass a stream of their own, not the legacy default stream."""
    N = W.ragged_counts(24, 64, 4096)
    d_w, d_u = _inputs(N, seed=300)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(2):
        d_anc = torch.full((d_w.numel(),), -7, dtype=torch.int32, device="cuda")
        pf.pf_systematic_resample_noalloc(N, d_w, d_u, d_anc, stream=s.cuda_stream)
        s.synchronize()
        assert np.array_equal(d_anc.cpu().numpy(), _with_caller_scratch(N, d_w, d_u, stream=s.cuda_stream))


def test_noalloc_rejects_sizes_beyond_its_array():
    hdr = open(__file__.replace("tests/test_zz_no_alloc.py", "include/pf.h")).read()
    max_p = int(hdr.split("#define PF_NOALLOC_MAX_PARTICLES")[1].split()[0])
    N = np.array([max_p // 2 + 1, max_p // 2 + 1], dtype=np.int32)
    d_w = torch.ones(int(N.sum()), dtype=torch.float64, device="cuda")
    d_u = torch.zeros(2, dtype=torch.float64, device="cuda")
    d_anc = torch.empty(int(N.sum()), dtype=torch.int32, device="cuda")
    with pytest.raises(pf.PFError) as e:
        pf.pf_systematic_resample_noalloc(N, d_w, d_u, d_anc)
    assert e.value.status == pf.PF_EINVAL and "PF_NOALLOC_MAX_PARTICLES" in str(e.value)
