"""The training step (a1-a6 through gem_forward / gem_backward) and the
optimiser step capture into one CUDA graph and replay with new inputs: no
call on the step's path synchronises or allocates once the context exists."""
import numpy as np
import pytest
import torch

import gemtest as gt
from paper_2509_25075_gb300 import binding
from paper_2509_25075_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

W = syn.Workload("graph", d=64, M=700, B=6, apix=1.2, seed=31)


def test_step_replays_from_a_cuda_graph():
    s = torch.cuda.Stream()
    torch.cuda.set_stream(s)
    try:
        ctx = binding.Context(W.d, W.apix, W.B, W.M, tau=W.tau, stream=s)
        first = gt.inputs(W)
        static = {k: gt.to_dev(v) for k, v in first.items()}
        loss = torch.zeros(1, dtype=torch.float64, device=gt.DEV)
        grad = torch.zeros(W.M, 11, device=gt.DEV)
        raw = static["params"].clone()
        m = torch.zeros_like(raw)
        v = torch.zeros_like(raw)
        params_out = torch.empty_like(raw)

        def step():
            ctx.gem_forward(static["params"], static["R"], static["t"], static["images"], loss,
                            ctf_params=static["ctf_params"])
            ctx.gem_backward(grad)
            ctx.gem_adam_step(raw, m, v, grad, params_out, (0.01, 0.0, 0.0, 0.0), 1)

        step()  # first use outside the capture
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            step()
        for seed in (41, 42):
            inp = gt.inputs(W, seed=seed)
            for k, t in static.items():
                t.copy_(torch.as_tensor(inp[k]))
            raw.copy_(static["params"])
            m.zero_()
            v.zero_()
            g.replay()
            s.synchronize()
            got_loss, got_grad, got_raw = loss.item(), grad.clone(), raw.clone()
            raw.copy_(static["params"])
            m.zero_()
            v.zero_()
            step()  # eager, same inputs
            s.synchronize()
            assert got_loss == loss.item()  # the forward is deterministic
            gt.assert_grad_close(got_grad.cpu().numpy(), grad.cpu().numpy().astype(np.float64),
                                 norm_tol=1e-6, entry_tol=1e-4)
            torch.testing.assert_close(got_raw, raw, rtol=1e-6, atol=1e-6)
        assert ctx.gem_status() == binding.GEM_OK
        ctx.close()
    finally:
        torch.cuda.set_stream(torch.cuda.default_stream())
