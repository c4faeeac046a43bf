"""pb_anneal_ea_noalloc: the EA +-1 anneal for callers that cannot allocate
device memory (code inside a memory arena it does not own, or loops where an
allocation, or the synchronisation it can cause, is not allowed).  Its scratch
is a fixed file-scope device array; inputs and outputs are the caller's device
buffers.  It must give exactly what pb_anneal gives (+-1 couplings: bit-exact),
call after call, although every call reuses the same scratch array, and it must
not wait for the GPU.  Collected last on purpose."""
import numpy as np
import pytest

import synth_inputs as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    from paper_2510_23419_gb300 import _build, native
    _build.build()
    native.load()
    return native


def _buffers(L, R):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    N = L ** 3
    return dict(best_E=torch.full((R,), float("nan"), dtype=torch.float64, device=dev),
                final_E=torch.full((R,), float("nan"), dtype=torch.float64, device=dev),
                best_sweep=torch.full((R,), -7, dtype=torch.int32, device=dev),
                best_state=torch.zeros((R, N), dtype=torch.int8, device=dev),
                final_state=torch.zeros((R, N), dtype=torch.int8, device=dev))


def _call(pb, L, Jd, sched, R, seed, b, stream):
    pb.pb_anneal_ea_noalloc(L, Jd.data_ptr(), sched, R, seed, b["best_E"].data_ptr(), b["best_sweep"].data_ptr(),
                            b["best_state"].data_ptr(), b["final_E"].data_ptr(), b["final_state"].data_ptr(),
                            stream=stream)


def _noalloc(pb, L, J, sched, R, seed):
    import torch
    Jd = torch.from_numpy(np.ascontiguousarray(J)).to(torch.device("cuda", torch.cuda.current_device()))
    b = _buffers(L, R)
    _call(pb, L, Jd, sched, R, seed, b, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in b.items()}


def test_noalloc_matches_pb_anneal_call_after_call(pb):
    # (L, R, S, seed): R = 13 and 37 leave a partial last replica quad
    cases = [(16, 64, 200, 5), (8, 24, 50, 6), (16, 64, 200, 5), (8, 13, 40, 9), (32, 8, 30, 7), (12, 37, 25, 3)]
    for L, R, S, seed in cases:
        J = syn.ea_couplings(L, "pm1", seed)
        sc = pb.make_schedule(pb.PB_SCHED_GEOMETRIC, S, 0.1, 5.0)
        a = _noalloc(pb, L, J, sc, R, seed)
        b = pb.anneal(pb.PB_TOPO_EA3D, J, sc, R, seed, L=L, form=pb.PB_FORM_RESIDENT)
        for k in ("best_E", "final_E", "best_sweep", "best_state", "final_state"):
            assert np.array_equal(a[k], b[k]), (L, R, S, k)


def test_noalloc_does_not_wait_for_the_gpu(pb):
    """The call only queues work: with a ~0.3 s spin queued before it on the same
    stream, the stream is still busy when the call returns."""
    import torch
    L, R = 8, 16
    J = syn.ea_couplings(L, "pm1", 2)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, 20, 0.1, 3.0)
    Jd = torch.from_numpy(J).cuda()
    _noalloc(pb, L, J, sc, R, 4)  # warm-up: the first call on a device may load the library's module
    b = _buffers(L, R)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        torch.cuda._sleep(600_000_000)  # bounded spin, about 0.3 s at 2 GHz
    _call(pb, L, Jd, sc, R, 4, b, s)
    busy = not s.query()
    s.synchronize()
    assert busy
    ref = pb.anneal(pb.PB_TOPO_EA3D, J, sc, R, 4, L=L, form=pb.PB_FORM_RESIDENT)
    assert np.array_equal(b["best_E"].cpu().numpy(), ref["best_E"])


def test_noalloc_reports_bad_couplings_in_outputs(pb):
    L, R = 8, 12
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, 10, 0.1, 1.0)
    for bad in (0, 2):
        J = syn.ea_couplings(L, "pm1", 3).copy()
        J[1, 17] = bad
        a = _noalloc(pb, L, J, sc, R, 1)
        assert np.all(a["best_sweep"] == pb.PB_NOALLOC_BAD_COUPLINGS)
        assert np.all(np.isnan(a["best_E"])) and np.all(np.isnan(a["final_E"]))
    # the flag does not leak into the next call on the shared array
    J = syn.ea_couplings(L, "pm1", 3)
    a = _noalloc(pb, L, J, sc, R, 1)
    b = pb.anneal(pb.PB_TOPO_EA3D, J, sc, R, 1, L=L, form=pb.PB_FORM_RESIDENT)
    assert np.array_equal(a["best_sweep"], b["best_sweep"]) and np.array_equal(a["best_E"], b["best_E"])


def test_noalloc_rejects_bad_shapes(pb):
    import torch
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    J = torch.zeros(3 * 34 ** 3, dtype=torch.int8, device="cuda")
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, 10, 0.1, 1.0)
    for L, want in ((7, pb.PB_ECOLOUR), (34, pb.PB_EINVAL), (0, pb.PB_EINVAL)):
        with pytest.raises(pb.PbError) as ei:
            pb.pb_anneal_ea_noalloc(L, J.data_ptr(), sc, 4, 1, out.data_ptr(), out.data_ptr(), out.data_ptr(),
                                    out.data_ptr(), out.data_ptr())
        assert ei.value.status == want, L


def test_noalloc_rejects_oversize(pb):
    import torch
    L, R = 32, 1024  # 2 * 1024 * 32768 bytes of state > 16 MiB
    J = torch.from_numpy(syn.ea_couplings(L, "pm1", 1)).cuda()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pb.PbError) as ei:
        pb.pb_anneal_ea_noalloc(L, J.data_ptr(), pb.make_schedule(pb.PB_SCHED_LINEAR, 10, 0.1, 1.0), R, 1,
                                out.data_ptr(), out.data_ptr(), out.data_ptr(), out.data_ptr(), out.data_ptr())
    assert ei.value.status == pb.PB_EINVAL
    assert "16777216" in str(ei.value)
