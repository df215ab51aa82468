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


def test_host_memory_is_rejected(env):
    pf, torch = env
    w = W.robertson(N=128, T=2)
    need = pf.pf_device_bytes(w.ode, w.d, w.p, 128)
    pinned = torch.empty(need + 512, dtype=torch.uint8, pin_memory=True)
    off = (-pinned.data_ptr()) % 256
    with pytest.raises(pf.PfError) as ei:
        pf.Filter.from_workload(w, N=128, device_buffer=(pinned.data_ptr() + off, need))
    assert ei.value.status == pf.PF_ERR_INVALID_ARG
    import numpy as np_
    host = np_.zeros(need + 512, dtype=np_.uint8)
    off = (-host.ctypes.data) % 256
    with pytest.raises(pf.PfError) as ei:
        pf.Filter.from_workload(w, N=128, device_buffer=(host.ctypes.data + off, need))
    assert ei.value.status == pf.PF_ERR_INVALID_ARG
