"""Failure handling without a device fault: a bounded device wait on a flag
that nothing sets gives up, reports BS_ERR_TIMEOUT through the status word,
and the context keeps working; host-side errors (bad arguments, undersized
budgets) are rejected before any launch."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2209_00220_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_00220_gb300 import build_lib
    build_lib.build()
    from paper_2209_00220_gb300 import bytestore
    return bytestore


def test_bounded_wait_gives_up_and_context_survives(B):
    assert B.bs_last_device_error() == 0
    assert B.bs_selftest_bounded_wait(1 << 12) is True
    assert B.bs_last_device_error() == B.BS_ERR_TIMEOUT
    assert B.bs_last_device_error() == 0  # read and cleared
    # the context still answers: a scan and lookup match the oracle
    v = synth.config_sweep_column(100003, 12, 1.0, 5)
    col = B.bs_encode_column(v, "ppvbs")
    a, _ = synth.pick_literals(v, "lt", 0.2, 1)
    bits = B.bs_scan(col, "lt", a)
    want = orc.scan_values(v, "lt", a)
    assert np.array_equal(bits[: want.size].cpu().numpy().view(np.uint32), want)
    vals, cnt = B.bs_lookup(col, bits)
    assert np.array_equal(vals[: int(cnt.item())].cpu().numpy(), orc.lookup(v, want))
    with pytest.raises(B.BsError):
        B.bs_selftest_bounded_wait(1 << 30)  # above the documented limit


def test_host_errors_are_rejected_before_launch(B):
    import torch
    v = synth.config_sweep_column(5000, 10, 1.0, 6)
    col = B.bs_encode_column(v, "ppvbs")
    with pytest.raises(B.BsError):
        B.lib()  # loaded
        B._check(B.lib().bs_scan(col.handle, 99, 0, 0, None, None), "bs_scan")  # bad op, no output
    with pytest.raises(B.BsError):
        B.bs_batch_create([{"preds": [(col, "lt", 1)] * 5, "out": torch.empty(8, dtype=torch.int32, device="cuda")}])
    srv = B.bs_server_create(max_batch=4, result_bytes=4096, scratch_bytes=1 << 20)
    with pytest.raises(B.BsError):
        srv.submit([(col, "ne", int(v[0]))])  # its result bound never fits 4 KB
    assert srv.stats()["rejected"] == 1
    srv.destroy()
    assert B.bs_last_device_error() == 0
