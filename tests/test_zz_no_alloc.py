"""lbib_mesh_measures_noalloc: the allocation-free volume and area
reduction, through the C ABI, against the volume and area lbib_get_body
reports for the same mesh.

Collected last on purpose: it must pass both alone in a fresh process (the
first call then does the per-device set-up) and after every other test.
"""
import numpy as np
import pytest

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


@pytest.mark.gpu
def test_noalloc_measures_match_lbib_get_body_on_two_calls_in_a_row(lbib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
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

    stream = torch.cuda.Stream(device=dev)
    dX = [torch.from_numpy(np.ascontiguousarray(X, dtype=np.float64)).to(dev) for X, _, _ in meshes]
    dT = [torch.from_numpy(np.ascontiguousarray(T, dtype=np.int32)).to(dev) for _, T, _ in meshes]
    out = [torch.full((2,), float("nan"), dtype=torch.float64, device=dev) for _ in meshes]
    torch.cuda.synchronize()
    for k in range(2):  # two calls in a row on one stream, no synchronisation between them
        lbib.lbib_mesh_measures_noalloc(dX[k], dX[k].shape[0], dT[k], dT[k].shape[0], out[k], stream.cuda_stream)
    stream.synchronize()
    for k, (_, _, body) in enumerate(meshes):
        vol, area = out[k].cpu().numpy()
        assert abs(vol - body["volume"]) <= 1e-12 * abs(body["volume"])
        assert abs(area - body["area"]) <= 1e-12 * abs(body["area"])
    assert abs(out[0][0].item() - out[1][0].item()) > 1.0  # different meshes, no stale result
