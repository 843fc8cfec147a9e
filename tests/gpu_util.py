"""Helpers shared by the GPU tests: run the CUDA path through the C ABI binding."""
import numpy as np


def to_numpy_u64(t):
    import torch
    return t.view(torch.int64).cpu().numpy().view(np.uint64)


def gpu_count(n, src, dst, k, stream=None):
    """Build the device graph, count, return uint64[n, C_k] numpy (and check status)."""
    import torch
    from paper_2201_11655_b300 import vdmc
    with vdmc.graph_create(n, src, dst, stream=stream) as g:
        out = vdmc.count(g, k, stream=stream)
        torch.cuda.synchronize()
        assert g.device_status() == 0
        return to_numpy_u64(out)


def gpu_count_roots(g, k, lo, hi):
    import torch
    from paper_2201_11655_b300 import vdmc
    out = vdmc.count_roots(g, k, lo, hi)
    torch.cuda.synchronize()
    assert g.device_status() == 0
    return to_numpy_u64(out)
