"""Failure path of the device-side waits, on the GPU, without a fault.

The tensor-core biclique kernel is the library's only kernel whose threads
wait on one another (TMA -> MMA -> epilogue through mbarriers).  Every wait is
bounded by the global timer; a wait that runs out records an error word, the
kernel skips its writes, releases its tensor memory and ends, and the host
reports PB_ETIMEOUT.  The test hook PB_FLAG_TEST_EXPIRE_WAITS makes the load
warp issue no loads, so the waits for operands have nothing to wait for and
run out after 2 ms.  Afterwards the same context must still produce the
oracle's bit-exact trajectories.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    from paper_2510_23419_gb300 import _build, native
    _build.build()
    native.load()
    return native


def test_tensor_waits_run_out_and_context_survives(pb, orc):
    n, R, S, seed = 256, 128, 2, 5
    J = pb.pb_generate_biclique(n, pb.PB_DIST_PM1, 3)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.35, 3.5)
    inst = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, J, None, n=n)
    try:
        t0 = time.perf_counter()
        run = pb.pb_anneal(inst, sc, R, seed,
                           pb.make_opts(pb.PB_FORM_TENSOR, flags=pb.PB_FLAG_TEST_EXPIRE_WAITS))
        try:
            status = pb.pb_wait(run, 60000)
            elapsed = time.perf_counter() - t0
            assert status == pb.PB_ETIMEOUT
            assert "device-side wait" in pb.pb_last_error()
            assert elapsed < 30.0  # 2 ms per expired wait, a handful of launches
            with pytest.raises(pb.PbError, match="PB_ETIMEOUT"):
                pb.pb_energy(run, R)
        finally:
            pb.pb_run_destroy(run)
    finally:
        pb.pb_instance_destroy(inst)

    # the context is intact: the same anneal without the hook matches the oracle bit for bit
    g = pb.anneal(pb.PB_TOPO_BICLIQUE, J, sc, R, seed, n=n, form=pb.PB_FORM_TENSOR)
    o = orc.anneal_biclique(n, J.astype(np.float64), None, orc.schedule(orc.SCHED_LINEAR, 0.35, 3.5, S), R, seed)
    for key in ("final_state", "best_state", "final_E", "best_E", "best_sweep"):
        assert np.array_equal(g[key], o[key]), key
