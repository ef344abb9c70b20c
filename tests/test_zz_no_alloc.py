"""lbib_mesh_measures_noalloc: the allocation-free volume and area
reduction, called through the C ABI.  Its results are compared with the FP64
oracle's volume and area of the same vertex positions (and with what
lbib_get_body, the allocating path, reports for them).

Collected last on purpose: it must pass both alone in a fresh process (the
first call then loads the library's device code) and after every other
test.
"""
import numpy as np
import pytest

import oracle
from paper_2207_06029_gb300 import workloads as W


@pytest.fixture(scope="module")
def lbib():
    from paper_2207_06029_gb300 import build, lbib as L
    build.build()
    L.load()
    return L


def test_sizes_beyond_the_maximum_are_rejected_before_any_cuda_call(lbib):
    with pytest.raises(lbib.LbibError) as ei:
        lbib.lbib_mesh_measures_noalloc(0, 3, 0, lbib.LBIB_NOALLOC_MAX_TRIS + 1, 0)
    assert ei.value.code == lbib.LBIB_ETOOBIG
    assert "LBIB_NOALLOC_MAX_TRIS" in str(ei.value)
    with pytest.raises(lbib.LbibError) as ei:
        lbib.lbib_mesh_measures_noalloc(0, 3, 0, -1, 0)
    assert ei.value.code == lbib.LBIB_EINVAL


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to("cuda:0")


@pytest.mark.gpu
def test_noalloc_measures_match_the_oracle_on_two_calls_in_a_row(lbib, cuda):
    torch = cuda
    torch.cuda.set_device(0)
    meshes = []
    # a rigid sphere of 20480 triangles (80 blocks of the reduction) ...
    v, f = W.icosphere(5, 8.0, (19.5, 19.5, 19.5))
    ctx = lbib.Context((40, 40, 40), 0.8, precision=lbib.LBIB_FP64)
    ctx.add_body(v, f, rigid=True, density_ratio=1.3, ref_radius=8.0, gravity=(0.0, 0.0, -1e-5),
                 u0=(1e-3, 0.0, 0.0), omega0=(0.0, 2e-4, 1e-4))
    ctx.step(3)
    meshes.append((ctx.markers(0)[0], f, ctx.body(0)))
    ctx.close()
    # ... then a deforming membrane of 1280 triangles (5 blocks), so the
    # second call must not see partial sums left by the first
    case = W.case_capsule_shear(n=28, tau=0.8, shear_rate=2e-3, radius=5.0, level=3, Ca=0.05, Eb=0.01,
                                kv=1.0, precision=W.PREC_FP64)
    ctx = lbib.Context.from_case(case)
    ctx.step(12)
    meshes.append((ctx.markers(0)[0], case.bodies[0].tris, ctx.body(0)))
    ctx.close()

    stream = torch.cuda.Stream(device="cuda:0")
    dX = [_dev(torch, X, np.float64) for X, _, _ in meshes]
    dT = [_dev(torch, T, np.int32) for _, T, _ in meshes]
    out = [torch.full((2,), float("nan"), dtype=torch.float64, device="cuda:0") for _ in meshes]
    torch.cuda.synchronize()
    for k in range(2):  # two calls in a row on one stream, no synchronisation between them
        lbib.lbib_mesh_measures_noalloc(dX[k], dX[k].shape[0], dT[k], dT[k].shape[0], out[k], stream.cuda_stream)
    stream.synchronize()
    for k, (X, T, body) in enumerate(meshes):
        vol, area = out[k].cpu().numpy()
        T32 = np.ascontiguousarray(T, dtype=np.int32)
        v_ref, a_ref = oracle.volume(X, T32), oracle.area(X, T32)
        assert abs(vol - v_ref) <= 1e-12 * abs(v_ref)
        assert abs(area - a_ref) <= 1e-12 * abs(a_ref)
        # the allocating path reports the same measures
        assert abs(vol - body["volume"]) <= 1e-12 * abs(v_ref)
        assert abs(area - body["area"]) <= 1e-12 * abs(a_ref)
    assert abs(out[0][0].item() - out[1][0].item()) > 1.0  # different meshes, no stale result


@pytest.mark.gpu
def test_noalloc_bad_index_gives_nan_and_empty_mesh_gives_zeros(lbib, cuda):
    """A vertex index equal to nv is skipped on the device and poisons both
    outputs; the next call (counter and flag cleared) is clean again, and a
    mesh without triangles measures zero."""
    torch = cuda
    torch.cuda.set_device(0)
    v, f = W.icosphere(2, 3.0, (0.0, 0.0, 0.0))
    bad = f.copy()
    bad[17, 1] = v.shape[0]
    dX = _dev(torch, v, np.float64)
    out = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    lbib.lbib_mesh_measures_noalloc(dX, v.shape[0], _dev(torch, bad, np.int32), bad.shape[0], out)
    torch.cuda.synchronize()
    assert np.isnan(out.cpu().numpy()).all()
    lbib.lbib_mesh_measures_noalloc(dX, v.shape[0], _dev(torch, f, np.int32), f.shape[0], out)
    torch.cuda.synchronize()
    T32 = np.ascontiguousarray(f, dtype=np.int32)
    vol, area = out.cpu().numpy()
    assert abs(vol - oracle.volume(v, T32)) <= 1e-12 * oracle.volume(v, T32)
    assert abs(area - oracle.area(v, T32)) <= 1e-12 * oracle.area(v, T32)
    out.fill_(float("nan"))
    empty = torch.zeros((0, 3), dtype=torch.int32, device="cuda:0")
    lbib.lbib_mesh_measures_noalloc(dX, v.shape[0], empty, 0, out)
    torch.cuda.synchronize()
    assert out.cpu().numpy().tolist() == [0.0, 0.0]


@pytest.mark.gpu
def test_noalloc_binding_rejects_wrong_tensors(lbib, cuda):
    """The binding refuses tensors the kernel would misread (int64 indices,
    float32 positions, host memory) before any CUDA call."""
    torch = cuda
    torch.cuda.set_device(0)
    v, f = W.icosphere(1, 2.0)
    dX = _dev(torch, v, np.float64)
    out = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    for X, T, o in [(dX, _dev(torch, f, np.int64), out),
                    (dX.float(), _dev(torch, f, np.int32), out),
                    (dX, torch.from_numpy(f.astype(np.int32)), out)]:
        with pytest.raises(lbib.LbibError) as ei:
            lbib.lbib_mesh_measures_noalloc(X, v.shape[0], T, f.shape[0], o)
        assert ei.value.code == lbib.LBIB_EINVAL
