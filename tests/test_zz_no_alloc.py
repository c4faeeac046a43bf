"""pb_anneal_ea_noalloc: the EA +-1 anneal for callers that cannot allocate
device memory (code inside a memory arena it does not own, or loops where an
allocation is not allowed).  Its scratch is a fixed file-scope device array;
inputs and outputs are the caller's device buffers.  It must give exactly what
pb_anneal gives (+-1 couplings: bit-exact), call after call, although every
call reuses the same scratch array.  Collected last on purpose."""
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


def _noalloc(pb, L, J, sched, R, seed):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    N = L ** 3
    Jd = torch.from_numpy(np.ascontiguousarray(J)).to(dev)
    bE = torch.full((R,), float("nan"), dtype=torch.float64, device=dev)
    fE = torch.full((R,), float("nan"), dtype=torch.float64, device=dev)
    bs = torch.full((R,), -7, dtype=torch.int32, device=dev)
    bst = torch.zeros((R, N), dtype=torch.int8, device=dev)
    fst = torch.zeros((R, N), dtype=torch.int8, device=dev)
    stream = torch.cuda.current_stream()
    pb.pb_anneal_ea_noalloc(L, Jd.data_ptr(), sched, R, seed, bE.data_ptr(), bs.data_ptr(), bst.data_ptr(),
                            fE.data_ptr(), fst.data_ptr(), stream=stream)
    torch.cuda.synchronize()
    return dict(best_E=bE.cpu().numpy(), final_E=fE.cpu().numpy(), best_sweep=bs.cpu().numpy(),
                best_state=bst.cpu().numpy(), final_state=fst.cpu().numpy())


def test_noalloc_matches_pb_anneal_call_after_call(pb):
    cases = [(16, 64, 200, 5), (8, 24, 50, 6), (16, 64, 200, 5), (32, 8, 30, 7)]
    for L, R, S, seed in cases:
        J = syn.ea_couplings(L, "pm1", seed)
        sc = pb.make_schedule(pb.PB_SCHED_GEOMETRIC, S, 0.1, 5.0)
        a = _noalloc(pb, L, J, sc, R, seed)
        b = pb.anneal(pb.PB_TOPO_EA3D, J, sc, R, seed, L=L, form=pb.PB_FORM_RESIDENT)
        for k in ("best_E", "final_E", "best_sweep", "best_state", "final_state"):
            assert np.array_equal(a[k], b[k]), (L, R, S, k)


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
