"""Allocation-free sampling entry point (kadabra_sample_static).

Some callers cannot allocate device memory once they are running: a service
that reserves all of its GPU memory at start-up and must not allocate while it
serves requests, or a plug-in whose host framework owns the device allocator.
kadabra_sample_static gives them the sampling kernel with its scratch in a
fixed array inside the library, so they only pass their graph and their own
output array.

These tests call it through the C ABI and require its counters to equal those
of kadabra_sample_epoch on the same sample indices, for two calls in a row
(the second call reuses the array the first one left behind), with the free
device memory unchanged across both calls, the first included: loading a
graph already reserved the array on the device.  The file is named so that
pytest collects it after every other test.
"""
import numpy as np
import pytest

from paper_1910_11039_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_11039_gb300 import build as B
    B.build()
    from paper_1910_11039_gb300 import kadabra
    kadabra.load()
    torch.cuda.set_device(0)
    return kadabra


@pytest.mark.parametrize("name,E", [("er2000", 3000), ("rmat14", 2500), ("grid64", 1500)])
def test_static_sampling_matches_sample_epoch(K, name, E):
    import torch
    g = I.config_graph(name)
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=0.005, delta=0.1, seed=5, n_calib=100)
    assert q.info().omega_ceil >= 2 * E
    q.sample_epoch(E)
    first_epoch = q.result(btilde=False)["counts"].copy()
    q.sample_epoch(E)
    two_epochs = q.result(btilde=False)["counts"].copy()

    counts = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free = [torch.cuda.mem_get_info()[0]]
    # call 1 (in a fresh process, the first call of the entry point): samples
    # [0, E) of the adaptive stream
    K.sample_static(G, 5, 1, 0, E, counts.data_ptr())
    free.append(torch.cuda.mem_get_info()[0])
    assert np.array_equal(counts.cpu().numpy().view(np.uint32), first_epoch)
    # call 2: samples [E, 2E) added to the same caller-owned array
    K.sample_static(G, 5, 1, E, E, counts.data_ptr())
    free.append(torch.cuda.mem_get_info()[0])
    assert np.array_equal(counts.cpu().numpy().view(np.uint32), two_epochs)
    assert free[0] == free[1] == free[2], free


def test_static_sampling_calibration_stream(K, orc):
    import torch
    g = I.config_graph("er2000")
    G = K.Graph.from_inputs(g)
    counts = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    for _ in range(2):
        counts.zero_()
        K.sample_static(G, 3, 0, 0, 700, counts.data_ptr())
        want, _ = orc.run_samples(g, 3, 0, 0, 700)
        assert np.array_equal(counts.cpu().numpy().view(np.uint32), want)


def test_static_sampling_rejects_graphs_beyond_the_array(K):
    import torch
    # a path of 3.5M vertices needs 126 MB per in-flight sample: more than the array
    n = 3_500_000
    deg = np.full(n, 2, dtype=np.int64)
    deg[0] = deg[-1] = 1
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=off[1:])
    cols = np.empty(off[-1], dtype=np.int32)
    left = np.arange(1, n)            # vertices with a left neighbour: first entry of their row
    right = np.arange(0, n - 1)
    cols[off[:-1][left]] = left - 1
    cols[off[1:][right] - 1] = right + 1   # right neighbour: last entry of the row
    G = K.Graph(n, off, cols, offsets_64=True, skip_validate=True)
    counts = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(K.KadabraError) as ei:
        K.sample_static(G, 1, 1, 0, 10, counts.data_ptr())
    assert ei.value.status == 1 and "static scratch" in str(ei.value)
