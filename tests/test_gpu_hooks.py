"""GPU: a world whose device memory and streams belong to PyTorch.

The world descriptor takes an allocator (alloc/free callbacks with a context pointer) and
the two CUDA streams to run on.  Here they are torch's caching allocator and two torch
streams, passed through the C ABI; the world must give the same bits as one that
allocates its own memory and creates its own streams, take every byte it uses from the
callbacks, and hand every byte back when it is destroyed."""
import numpy as np
import pytest

from paper_2311_04648_gb300 import dem, workloads as W

pytestmark = pytest.mark.gpu


def _scene():
    return W.dense_lattice(n=1500, seed=31, vel_sigma=0.3)


@pytest.mark.parametrize("precision,schedule", [("voxel_fp32", "velocity_bound"), ("fp64", "every_step")])
def test_world_on_torch_memory_and_streams_matches_a_self_allocating_world(precision, schedule):
    torch = pytest.importorskip("torch")
    dev = torch.cuda.current_device()
    sf = torch.cuda.Stream(device=dev, priority=-1)      # force / integration
    sd = torch.cuda.Stream(device=dev)                   # detection
    live = {}

    def alloc(nbytes):
        p = torch.cuda.caching_allocator_alloc(nbytes, device=dev, stream=sf)
        live[int(p)] = nbytes
        return int(p)

    def free(ptr):
        live.pop(int(ptr))
        torch.cuda.caching_allocator_delete(int(ptr))

    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated(dev)
    scene = _scene()
    a = dem.World.from_scene(scene, precision=precision, schedule=schedule, device=dev,
                             stream=sf.cuda_stream, detect_stream=sd.cuda_stream, alloc=alloc, free=free)
    b = dem.World.from_scene(scene, precision=precision, schedule=schedule, device=dev)
    try:
        assert a.stream() == sf.cuda_stream
        assert len(live) > 10
        assert torch.cuda.memory_allocated(dev) - before >= sum(live.values())
        for _ in range(3):
            a.step(100)
            b.step(100)
            for xa, xb in zip(a.owner_state(), b.owner_state()):
                assert np.array_equal(xa, xb)
        ca, cb = a.contacts(), b.contacts()
        assert len(ca["i"]) > 100
        for k in ca:
            assert np.array_equal(ca[k], cb[k]), k
        sa, sb = a.stats(), b.stats()
        assert sa["rebuilds"] == sb["rebuilds"] and sa["steps"] == sb["steps"] == 300
    finally:
        a.close()
        b.close()
    assert live == {}                       # every allocation was handed back
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated(dev) == before


def test_owner_state_into_pinned_host_buffers_equals_the_copied_state():
    # pinned caller buffers are written by the device across the host link; pageable ones
    # through device scratch and copies: the same values, on ragged ranges (not a whole
    # number of 256-owner blocks) and at an interior address of a pinned allocation
    torch = pytest.importorskip("torch")
    w = dem.World.from_scene(_scene(), precision="voxel_fp32", schedule="velocity_bound")
    try:
        w.step(60)
        for first, n in ((0, w.n_owner), (37, 1000), (w.n_owner - 1, 1)):
            ref = w.owner_state(first, n)
            pads = []
            for c in (3, 4, 3, 3):
                t = torch.full((n + 5, c), np.nan, dtype=torch.float64).pin_memory()
                pads.append(t.numpy())
            out = tuple(p[5:] for p in pads)          # interior of the pinned block
            got = w.owner_state(first, n, out=out)
            for a, b, p in zip(ref, got, pads):
                assert np.array_equal(a, b)
                assert np.isnan(p[:5]).all()          # nothing written before the range
    finally:
        w.close()
