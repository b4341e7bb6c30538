"""The allocation-free extraction entry point (yf_sparams_noalloc) against yf_sparams.

yf_sparams stages its inputs and its S* intermediate in memory it allocates per call.
yf_sparams_noalloc serves callers that cannot allocate on the GPU (work enqueued during a
global-mode stream capture, or programs whose device memory belongs to their own pool):
they pass device buffers for every input and output, and the library keeps its one
intermediate in a fixed per-GPU array.  Here torch, acting as such a caller, owns all
buffers; two calls in a row with different port counts and frequency grids must both
reproduce the allocating entry point within the extraction tests' tolerance, also when
the call is captured into a CUDA graph in global mode and replayed on new inputs.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _spectra(seed, N, F):
    rng = np.random.default_rng(seed)
    freqs = np.linspace(1e9, 60e9, F)
    Vi = rng.normal(size=(N, F)) + 1j * rng.normal(size=(N, F))
    Zp = np.linspace(25.0, 90.0, N)[:, None] + 1j * rng.normal(size=(N, F))
    Ii = Vi / Zp
    Vt = Vi[:, None, :] * (0.3 * (rng.normal(size=(N, N, F)) + 1j * rng.normal(size=(N, N, F))))
    return freqs, Vi, Ii, Vt


def _dev(a):
    import torch
    a = np.asarray(a)
    if np.iscomplexobj(a):
        a = np.stack([a.real, a.imag], axis=-1)
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _cplx(t):
    a = t.cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


def _call_noalloc(yf, freqs, Vi, Ii, Vt):
    import torch
    N, F = Vi.shape
    S = torch.zeros((F, N, N, 2), dtype=torch.float64, device="cuda")
    Ss = torch.zeros_like(S)
    Zr = torch.zeros((N, F, 2), dtype=torch.float64, device="cuda")
    Zc = torch.zeros((F, 2), dtype=torch.float64, device="cuda")
    tau = torch.zeros((F, N, N), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    yf.sparams_noalloc(N, F, _dev(freqs), _dev(Vi), _dev(Ii), _dev(Vt), S, Zr, S_star=Ss,
                       Zc=Zc if N == 2 else None, tau=tau, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    return dict(S=_cplx(S), S_star=_cplx(Ss), Zr=_cplx(Zr), Zc=_cplx(Zc) if N == 2 else None,
                tau=tau.cpu().numpy())


def _close(a, b, rel=1e-12):
    return np.max(np.abs(a - b)) <= rel * max(np.max(np.abs(b)), 1e-300)


def test_noalloc_extraction_matches_allocating_entry_point(gpu):
    import torch
    torch.cuda.init()
    for seed, N, F in ((11, 3, 40), (12, 2, 64)):
        freqs, Vi, Ii, Vt = _spectra(seed, N, F)
        ref = gpu.sparams(freqs, Vi, Ii, Vt)
        got = _call_noalloc(gpu, freqs, Vi, Ii, Vt)
        for key in ("S_star", "S", "Zr", "tau"):
            assert _close(got[key], ref[key]), key
        if N == 2:
            assert _close(got["Zc"], ref["Zc"])


def test_noalloc_extraction_skips_optional_outputs(gpu):
    """S_star and tau (and Zc of a 2-port) are optional: passing None leaves S and Zr as the
    allocating entry point gives them."""
    import torch
    freqs, Vi, Ii, Vt = _spectra(13, 2, 48)
    ref = gpu.sparams(freqs, Vi, Ii, Vt)
    S = torch.zeros((48, 2, 2, 2), dtype=torch.float64, device="cuda")
    Zr = torch.zeros((2, 48, 2), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    gpu.sparams_noalloc(2, 48, _dev(freqs), _dev(Vi), _dev(Ii), _dev(Vt), S, Zr,
                        stream=stream.cuda_stream)
    torch.cuda.synchronize()
    assert _close(_cplx(S), ref["S"]) and _close(_cplx(Zr), ref["Zr"])


def test_noalloc_extraction_inside_a_captured_graph(gpu):
    """The reason the entry point exists: it can be enqueued while a stream is captured in
    global mode, where allocating is illegal.  One call is captured into a CUDA graph after
    an eager call on the same device; the graph is then replayed on new spectra copied into
    the same input buffers, twice, and each replay matches the allocating entry point."""
    import torch
    N, F = 3, 40
    freqs, Vi, Ii, Vt = _spectra(21, N, F)
    bufs = [_dev(freqs), _dev(Vi), _dev(Ii), _dev(Vt)]
    S = torch.zeros((F, N, N, 2), dtype=torch.float64, device="cuda")
    Ss = torch.zeros_like(S)
    Zr = torch.zeros((N, F, 2), dtype=torch.float64, device="cuda")
    tau = torch.zeros((F, N, N), dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        gpu.sparams_noalloc(N, F, *bufs, S, Zr, S_star=Ss, tau=tau, stream=side.cuda_stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="global"):
        cap = torch.cuda.current_stream()
        gpu.sparams_noalloc(N, F, *bufs, S, Zr, S_star=Ss, tau=tau, stream=cap.cuda_stream)
    for seed in (22, 23):
        freqs, Vi, Ii, Vt = _spectra(seed, N, F)
        for b, new in zip(bufs, (freqs, Vi, Ii, Vt)):
            b.copy_(_dev(new))
        S.zero_(); Ss.zero_(); Zr.zero_(); tau.zero_()
        graph.replay()
        torch.cuda.synchronize()
        ref = gpu.sparams(freqs, Vi, Ii, Vt)
        got = dict(S=_cplx(S), S_star=_cplx(Ss), Zr=_cplx(Zr), tau=tau.cpu().numpy())
        for key in ("S_star", "S", "Zr", "tau"):
            assert _close(got[key], ref[key]), (seed, key)


def test_noalloc_rejects_requests_beyond_its_scratch(gpu):
    import torch
    N, F = 8, 1024            # 8 * 8 * 1024 = 65536 > 32768 scratch entries
    dummy = torch.zeros(2 * N * N * F, dtype=torch.float64, device="cuda")
    with pytest.raises(gpu.YFError) as e:
        gpu.sparams_noalloc(N, F, dummy, dummy, dummy, dummy, dummy, dummy)
    assert e.value.code == gpu.E_INVALID
    assert "scratch" in str(e.value)
