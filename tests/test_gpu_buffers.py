"""pf_create_with_buffers: a filter laid out in caller-owned device memory (a
torch tensor here) runs exactly as one the library allocates, and the memory
stays the caller's after pf_destroy."""
import numpy as np
import pytest

from paper_1411_1702_gb300 import build as B
from paper_1411_1702_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    B.build()
    from paper_1411_1702_gb300 import pf
    pf.load()
    return pf, torch


@pytest.mark.parametrize("name,N", [("robertson", 3001), ("brusselator", 257), ("advdiff20", 40)])
def test_caller_buffer_filter_equals_library_filter(env, name, N):
    pf, torch = env
    w = W.get(name, N=N)
    need = pf.pf_device_bytes(w.ode, w.d, w.p, N)
    buf = torch.full((need + 4096,), 0xA5, dtype=torch.uint8, device="cuda")
    assert buf.data_ptr() % 256 == 0
    a = pf.Filter.from_workload(w, N=N)
    b = pf.Filter.from_workload(w, N=N, device_buffer=buf)
    for k in range(4):
        a.pf_assimilate(w.t_obs[k], w.y_obs[k])
        b.pf_assimilate(w.t_obs[k], w.y_obs[k])
    ea, eb = a.pf_get_ensemble(), b.pf_get_ensemble()
    for key in ea:
        assert np.array_equal(ea[key], eb[key]), key
    for u, v in zip(a.pf_estimates(), b.pf_estimates()):
        assert np.array_equal(u, v)
    # the filter wrote only inside what pf_device_bytes reported
    torch.cuda.synchronize()
    assert bool((buf[need:] == 0xA5).all())
    b.close()
    a.close()
    # still the caller's: usable after pf_destroy
    buf.fill_(7)
    torch.cuda.synchronize()
    assert int(buf[:64].sum()) == 7 * 64
