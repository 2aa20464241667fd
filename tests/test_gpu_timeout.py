"""The bounded wait for table copies, run out on purpose (no fault, no
hang): with a wait budget of zero every block gives up before it looks,
waits (bounded) for its copies to land, skips its terms and marks the
result; every host entry point reports ZXP_ETIMEDOUT and the device result
carries flags bit 1.  With the default budget restored the same context
gives the exact value again."""
import pytest

import paper_2403_06777_gb300 as Z
import zxp_inputs as zi

pytestmark = pytest.mark.gpu


def test_wait_budget_runs_out_and_reports_timeout():
    import torch
    assert torch.cuda.is_available(), "this test needs a GPU"
    ctx = Z.zxp_ctx_create(0)
    try:
        w = zi.workload_medium(0)
        s = Z.zxp_compile(w.gates, w.n, w.out_bits)
        n = 1 << s.info["k"]
        ws = Z.zxp_compile(zi.workload_large(0).gates, 50, zi.workload_large(0).out_bits)
        ref, ref_w = Z.zxp_amplitude(ctx, s), Z.zxp_eval(ctx, ws, 0, 1 << 20)
        try:
            Z.zxp_set_wait_budget(0)
            for f in (lambda: Z.zxp_eval(ctx, s, 0, n), lambda: Z.zxp_eval(ctx, s, 5, 1000),
                      lambda: Z.zxp_amplitude(ctx, s), lambda: Z.zxp_eval(ctx, ws, 0, 1 << 20),
                      lambda: Z.zxp_eval_wide(ctx, s, 0, n),
                      lambda: Z.zxp_poll(ctx, Z.zxp_submit(ctx, s), -1)):
                with pytest.raises(Z.ZxpError) as e:
                    f()
                assert e.value.code == Z.ZXP_ETIMEDOUT
            out = torch.zeros(5, dtype=torch.int64, device="cuda")
            Z.zxp_eval_device(ctx, s, 0, n, out.data_ptr())
            torch.cuda.synchronize()
            assert (out[4].item() >> 32) & 2
        finally:
            Z.zxp_set_wait_budget(-1)
        assert Z.zxp_amplitude(ctx, s) == ref
        assert Z.zxp_eval(ctx, ws, 0, 1 << 20) == ref_w
    finally:
        ctx.close()


def test_wait_budget_bounds():
    with pytest.raises(Z.ZxpError) as e:
        Z.zxp_set_wait_budget(1 << 40)
    assert e.value.code == Z.ZXP_EINVAL
    Z.zxp_set_wait_budget(-1)
