"""The bounded wait for table copies, run out on purpose (no fault, no
hang): with zxp_test_table_timeout on, every launch's barrier expects 16
bytes more than its copies deliver, so every block's wait runs to its limit,
gives up, skips its terms and marks the result; the host entry points report
ZXP_ETIMEDOUT and the device result carries flags bit 1.  Each such launch
ends within the wait's bound.  With the setting off again the same context
gives the exact values again."""
import time

import pytest

import paper_2403_06777_gb300 as Z
import zxp_inputs as zi

pytestmark = pytest.mark.gpu
WAIT_BOUND_S = 5.0


def test_table_wait_runs_out_and_reports_timeout():
    import torch
    assert torch.cuda.is_available(), "this test needs a GPU"
    ctx = Z.zxp_ctx_create(0)
    try:
        w = zi.workload_medium(0)
        s = Z.zxp_compile(w.gates, w.n, w.out_bits)
        n = 1 << s.info["k"]
        wl = zi.workload_large(0)
        sl = Z.zxp_compile(wl.gates, wl.n, wl.out_bits)   # inner parameters
        ref, ref_l = Z.zxp_amplitude(ctx, s), Z.zxp_eval(ctx, sl, 0, 1 << 20)
        ref_w = Z.zxp_eval_wide(ctx, s, 0, n)
        secs = []
        try:
            Z.zxp_test_table_timeout(True)
            for f in (lambda: Z.zxp_eval(ctx, s, 5, 1000), lambda: Z.zxp_eval(ctx, sl, 0, 1 << 20),
                      lambda: Z.zxp_eval_wide(ctx, s, 0, n),
                      lambda: Z.zxp_poll(ctx, Z.zxp_submit(ctx, s), -1)):
                t = time.perf_counter()
                with pytest.raises(Z.ZxpError) as e:
                    f()
                secs.append(time.perf_counter() - t)
                assert e.value.code == Z.ZXP_ETIMEDOUT
            out = torch.zeros(5, dtype=torch.int64, device="cuda")
            Z.zxp_eval_device(ctx, s, 0, n, out.data_ptr())
            torch.cuda.synchronize()
            assert (out[4].item() >> 32) & 2
        finally:
            Z.zxp_test_table_timeout(False)
        print("timed-out launches took", ["%.2f s" % x for x in secs])
        assert max(secs) < WAIT_BOUND_S
        assert Z.zxp_amplitude(ctx, s) == ref
        assert Z.zxp_eval(ctx, sl, 0, 1 << 20) == ref_l
        assert Z.zxp_eval_wide(ctx, s, 0, n) == ref_w
    finally:
        ctx.close()
