"""GPU parity of the Table V reconstruction (through the C ABI) against the
FP64 oracle after a fixed number of iterations (tolerance 1e-4 relative L2 on
the reconstructed volume), plus checkpoint/resume and frame independence."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import camera as O
from oracle import recon as OR
from paper_1812_03358_b300 import build, inputs as I, lt

pytestmark = pytest.mark.gpu

TOL = 1e-4


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lt.lib()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def ops_for(vol, cams):
    return [(lambda v, c=c: O.forward(vol, c, v).ravel(), lambda r, c=c: O.adjoint(vol, c, r).ravel())
            for c in cams]


def measure(vol, cams, x_true, scales=None):
    ys = [O.forward(vol, c, x_true).ravel() for c in cams]
    if scales:
        ys = [y / s for y, s in zip(ys, scales)]
    return ys


def run_gpu(vol, cams, ys, n_iter, ws=None, **kw):
    plan = lt.Plan(vol, cams)
    y = dev(np.concatenate(ys)).reshape(1, -1)
    w = dev(np.concatenate(ws)).reshape(1, -1) if ws is not None else None
    rec = lt.Recon(plan, y, w=w, **kw)
    rec.iterate(n_iter)
    x, gains, fit = rec.get()
    return host(x)[0], gains[0], fit[0], rec, plan


def test_single_lens_50_iterations_match_oracle():
    vol, cam = I.config_single_small()
    x_true = I.gaussian_blobs(vol, seed=1000)
    ys = measure(vol, [cam], x_true)
    xg, gains, fit, _, _ = run_gpu(vol, [cam], ys, 50)
    ref = OR.fista(ops_for(vol, [cam]), ys, [None], vol.shape, 50, history=True)
    assert rel_l2(xg, ref["x"]) < TOL, rel_l2(xg, ref["x"])
    assert abs(fit - ref["fits"][-1]) <= TOL * ref["fits"][-1]


# rows of 20 voxels take the four-voxels-per-thread update, rows of 19 the
# one-voxel-per-thread update; ragged y and z in both
@pytest.mark.parametrize("psi,nx", [(0, 20), (1, 20), (1, 19)])
def test_regularised_weighted_l1_iterations_match_oracle(psi, nx):
    vol = I.Volume(nx, 18, 12, 4.0, 4.0, 5.0)
    cam = I.table_single_lens(40, 0.2, ks=2, kt=2)
    x_true = I.gaussian_blobs(vol, seed=1003)
    ys = measure(vol, [cam], x_true)
    ws = [I.uniform_random(cam.m, seed=99, lo=0.5, hi=1.5)]
    kw = dict(beta=2e-4, nu=1e-5, psi=psi, psi_delta=0.05)
    xg, _, _, _, _ = run_gpu(vol, [cam], ys, 30, ws=ws, **kw)
    ref = OR.fista(ops_for(vol, [cam]), ys, ws, vol.shape, 30, beta=2e-4, nu=1e-5, psi=psi, delta=0.05)
    assert rel_l2(xg, ref["x"]) < TOL, rel_l2(xg, ref["x"])


def test_two_cameras_with_gain_estimation():
    vol = I.Volume(16, 16, 16, 5.0, 5.0, 5.0)
    cams = [I.table_single_lens(36, 0.25), I.table_single_lens(30, 0.3, ks=2, kt=2)]
    x_true = I.gaussian_blobs(vol, seed=1004)
    ys = measure(vol, cams, x_true, scales=[1.0, 2.5])
    xg, gains, _, _, _ = run_gpu(vol, cams, ys, 40)
    ref = OR.fista(ops_for(vol, cams), ys, [None, None], vol.shape, 40)
    assert rel_l2(xg, ref["x"]) < TOL
    assert abs(gains[1] - ref["gains"][1]) < TOL * abs(ref["gains"][1])
    assert gains[0] == 1.0


def test_plenoptic_tiny_iterations_match_oracle():
    vol, cam = I.tiny_plenoptic()
    x_true = I.gaussian_blobs(vol, seed=1005)
    ys = measure(vol, [cam], x_true)
    xg, _, _, _, _ = run_gpu(vol, [cam], ys, 25)
    ref = OR.fista(ops_for(vol, [cam]), ys, [None], vol.shape, 25)
    assert rel_l2(xg, ref["x"]) < TOL


def test_plenoptic_full_size_two_iterations():
    vol, cam = I.config_plenoptic()
    x_true = I.plume_field(vol, seed=2000)
    y = I.poisson_images(O.forward(vol, cam, x_true), 1e4, seed=2001).astype(np.float64).ravel()
    xg, _, _, _, _ = run_gpu(vol, [cam], [y], 2)
    ref = OR.fista(ops_for(vol, [cam]), [y], [None], vol.shape, 2)
    assert rel_l2(xg, ref["x"]) < TOL


def test_checkpoint_resume_is_bit_identical():
    vol, cam = I.config_single_small()
    ys = measure(vol, [cam], I.gaussian_blobs(vol, seed=1000))
    _, _, _, rec, plan = run_gpu(vol, [cam], ys, 10, beta=1e-4)
    state = rec.state()
    rec.iterate(7)
    xa = host(rec.get()[0])
    rec2 = lt.Recon(plan, dev(ys[0]).reshape(1, -1), beta=1e-4)
    rec2.load_state(state)
    assert rec2.iterations == 10
    rec2.iterate(7)
    xb = host(rec2.get()[0])
    assert np.array_equal(xa, xb)


def test_frames_are_independent_problems():
    vol, cam = I.config_single_small()
    y0 = measure(vol, [cam], I.gaussian_blobs(vol, seed=1000))[0]
    y1 = measure(vol, [cam], I.gaussian_blobs(vol, seed=1001))[0]
    plan2 = lt.Plan(vol, [cam], frames=2)
    rec = lt.Recon(plan2, dev(np.stack([y0, y1])))
    rec.iterate(12)
    x2 = host(rec.get()[0])
    for f, y in enumerate([y0, y1]):
        xf, _, _, _, _ = run_gpu(vol, [cam], [y], 12)
        assert np.array_equal(x2[f], xf)


def test_async_result_read_matches_synchronous_read():
    vol = I.Volume(16, 16, 16, 5.0, 5.0, 5.0)
    cams = [I.table_single_lens(36, 0.25), I.table_single_lens(30, 0.3, ks=2, kt=2)]
    ys = measure(vol, cams, I.gaussian_blobs(vol, seed=1004), scales=[1.0, 2.5])
    plan = lt.Plan(vol, cams)
    rec = lt.Recon(plan, dev(np.concatenate([np.ravel(y) for y in ys])), estimate_gains=True)
    out = torch.empty(1 * (len(cams) + 1), dtype=torch.float64).pin_memory()
    rec.get_async(out)                       # before any iteration: fit 0, the initial gains
    _, gains0, fit0 = rec.get()
    torch.cuda.synchronize()
    assert out[0].item() == fit0[0] == 0.0 and np.array_equal(out[1:].numpy(), np.ravel(gains0))
    rec.iterate(7)
    rec.get_async(out)
    _, gains, fit = rec.get()
    torch.cuda.synchronize()
    assert abs(out[0].item() - fit[0]) <= 1e-12 * abs(fit[0])
    assert np.array_equal(out[1:].numpy(), np.ravel(gains))
    with pytest.raises(ValueError):
        rec.get_async(torch.empty(3, dtype=torch.float64))   # not page-locked
    # the C entry point itself takes pageable memory too (filled by a copy
    # instead of the kernel's write through the device mapping)
    pageable = np.zeros(len(cams) + 1)
    lt.lt_recon_get_async(rec.handle, pageable.ctypes.data, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert np.array_equal(pageable, out.numpy())


def test_set_data_from_unaligned_buffers_matches_aligned():
    """lt_recon_set_data copies the measurements and weights on the device
    (vector copies where both pointers are 16-byte aligned, element copies
    otherwise): data handed over from a buffer 4 bytes past an aligned
    address gives the same iterates, bit for bit, as the aligned original."""
    vol, cam = I.config_single_small()
    y = dev(measure(vol, [cam], I.gaussian_blobs(vol, seed=1005))[0]).reshape(1, -1)
    w = torch.rand(y.shape, device="cuda", generator=torch.Generator(device="cuda").manual_seed(7)) + 0.5
    plan = lt.Plan(vol, [cam])
    ybuf = torch.zeros(y.numel() + 1, device="cuda")
    wbuf = torch.zeros(w.numel() + 1, device="cuda")
    ybuf[1:].copy_(y.ravel())
    wbuf[1:].copy_(w.ravel())
    ref = lt.Recon(plan, torch.zeros_like(y), w=torch.ones_like(w))
    odd = lt.Recon(plan, torch.zeros_like(y), w=torch.ones_like(w))
    ref.set_data(y, w)
    odd.set_data(ybuf[1:].reshape(1, -1), wbuf[1:].reshape(1, -1))
    ref.iterate(6)
    odd.iterate(6)
    xa, ga, fa = ref.get()
    xb, gb, fb = odd.get()
    torch.cuda.synchronize()
    assert torch.equal(xa, xb) and np.array_equal(fa, fb) and np.array_equal(ga, gb)
