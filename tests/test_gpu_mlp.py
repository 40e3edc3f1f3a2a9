"""The selector network's CUDA kernels against the FP64 oracle (oracle/mlp.py):
forward values, loss, gradients (analytic backprop in FP64 on the same FP16
working weights) and Adam steps."""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu
F, H, C, B = 23, 128, 5, 96


def _setup(seed=0):
    import torch
    from paper_1307_2100_gb300 import tc
    rng = np.random.default_rng(seed)
    net = tc.tc_mlp_create(F, H, C, 256)
    n = tc.tc_mlp_num_params(net)
    assert n == mlp.n_params(F, H, C)
    theta = rng.normal(0, 0.2, n).astype(np.float32)
    tc.tc_mlp_set_params(net, theta.ctypes.data, n)
    work = np.empty(n, np.float32)
    tc.tc_mlp_get_params(net, work.ctypes.data, n, working=True)
    np.testing.assert_array_equal(work, theta.astype(np.float16).astype(np.float32))
    X = rng.normal(0, 1, (B, F)).astype(np.float32)
    T = rng.normal(0, 1, (B, C)).astype(np.float32)
    mask = (rng.uniform(size=(B, C)) > 0.25).astype(np.float32)
    dev = torch.device("cuda:0")
    return net, n, work, [torch.from_numpy(a).to(dev) for a in (X, T, mask)], (X, T, mask)


def test_forward_loss_and_gradients_match_fp64_oracle():
    import torch
    from paper_1307_2100_gb300 import tc
    net, n, work, (dX, dT, dM), (X, T, mask) = _setup()
    try:
        dev = dX.device
        Y = torch.empty(B, C, device=dev)
        tc.tc_mlp_forward(net, dX.data_ptr(), Y.data_ptr(), B)
        loss = torch.empty(1, device=dev)
        grad = torch.empty(n, device=dev)
        tc.tc_mlp_loss_grad(net, dX.data_ptr(), dT.data_ptr(), dM.data_ptr(), B, loss.data_ptr(),
                            grad.data_ptr())
        torch.cuda.synchronize()
        y_ref, _ = mlp.forward(work, X, F, H, C)
        np.testing.assert_allclose(Y.cpu().numpy(), y_ref, rtol=1e-4, atol=1e-4)
        L_ref, g_ref = mlp.loss_grad(work, X, T, mask, F, H, C)
        assert abs(loss.item() - L_ref) <= 1e-5 * max(1.0, abs(L_ref))
        g = grad.cpu().numpy().astype(np.float64)
        # FP32 accumulation against FP64: relative to the gradient's scale
        assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    finally:
        tc.tc_mlp_destroy(net)


def test_adam_steps_match_fp64_oracle_and_reduce_loss():
    import torch
    from paper_1307_2100_gb300 import tc
    net, n, work, (dX, dT, dM), (X, T, mask) = _setup(1)
    try:
        dev = dX.device
        loss = torch.empty(1, device=dev)
        grad = torch.empty(n, device=dev)
        master = np.empty(n, np.float32)
        tc.tc_mlp_get_params(net, master.ctypes.data, n, working=False)
        theta = master.astype(np.float64)
        m = np.zeros(n)
        v = np.zeros(n)
        losses = []
        for t in range(1, 31):
            tc.tc_mlp_loss_grad(net, dX.data_ptr(), dT.data_ptr(), dM.data_ptr(), B,
                                loss.data_ptr(), grad.data_ptr())
            tc.tc_mlp_adam_step(net, grad.data_ptr(), 1e-3, 0.9, 0.999, 1e-8, t)
            torch.cuda.synchronize()
            losses.append(loss.item())
            if t <= 3:   # one step of the oracle from the same gradient
                g = grad.cpu().numpy().astype(np.float64)
                theta, m, v = mlp.adam(theta, g, m, v, t, 1e-3)
                tc.tc_mlp_get_params(net, master.ctypes.data, n, working=False)
                np.testing.assert_allclose(master, theta, rtol=1e-5, atol=1e-6)
                theta = master.astype(np.float64)
        assert losses[-1] < losses[0]
    finally:
        tc.tc_mlp_destroy(net)
