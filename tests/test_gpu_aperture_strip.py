"""Every aperture of one image in one strip launch (cov_estimate_apertures)
against the oracle on each extracted aperture: complex64 within 1e-5
relative Frobenius, exact on small integers with COV_SUM, exact Hermitian
symmetry, agreement with the batched plan's forms, every element of R
overwritten, graph capture, and sampled apertures of the 1015 x 1015 image
(100 x 100 apertures of 25 x 25, 10 x 10 window)."""
import numpy as np
import pytest
import torch

import cov_workloads as wl
import paper_1303_2285_gb300 as cov

pytestmark = pytest.mark.gpu

from gpu_util import rel_fro  # noqa: E402

F32_TOL = 1e-5

SHAPES = [  # H, W, aperture, step, P, Q
    (64, 80, (25, 25), (10, 10), 10, 10),
    (47, 51, (20, 17), (9, 5), 4, 3),
    (40, 40, (40, 40), (1, 1), 16, 16),      # one aperture, the largest window
    (30, 70, (12, 30), (3, 7), 5, 9),
    (20, 130, (8, 64), (4, 33), 3, 1),       # 64-column apertures, one a CTA
    (33, 33, (9, 9), (8, 8), 1, 1),
    (26, 60, (26, 20), (1, 3), 16, 2),       # box of one row
    (35, 45, (11, 13), (2, 4), 6, 13),       # box of one column
    (64, 64, (64, 64), (1, 1), 16, 16),      # the largest aperture
    (90, 300, (16, 16), (16, 16), 8, 8),     # apertures side by side, no overlap
    (70, 200, (25, 25), (3, 2), 7, 10),      # many apertures a strip (step 2)
    (20, 40, (20, 20), (2, 2), 16, 4),       # fewer box rows than output rows (kept products from the walk)
]


def split(img_np, ap, step):
    H, W = img_np.shape
    nr, nc = (H - ap[0]) // step[0] + 1, (W - ap[1]) // step[1] + 1
    return nr, nc, lambda a, b: img_np[a * step[0]:a * step[0] + ap[0], b * step[1]:b * step[1] + ap[1]]


@pytest.mark.parametrize("H,W,ap,step,P,Q", SHAPES)
def test_strip_matches_oracle(oracle_mod, H, W, ap, step, P, Q):
    img_np = wl.complex_normal((H, W + 5), 40 + H + W, dtype="c64")  # ld = W + 5
    img = torch.from_numpy(img_np).cuda()[:, :W]
    nr, nc, sub = split(img_np[:, :W], ap, step)
    for norm in ("mean", "sum"):
        out = torch.full((nr * nc, P * Q, P * Q), complex(np.nan, np.nan), dtype=torch.complex64,
                         device="cuda")
        R = cov.apertures(img, ap, step, P, Q, norm=norm, out=out)
        torch.cuda.synchronize()
        got = R.cpu().numpy()
        assert np.isfinite(got.view(np.float32)).all()  # every element written
        for a in range(nr):
            for b in range(nc):
                want = oracle_mod.cov_window(sub(a, b).astype(np.complex128), P, Q,
                                             mean=(norm == "mean"))
                G = got[a * nc + b]
                assert rel_fro(G, want) < F32_TOL, (a, b, norm)
                assert np.array_equal(G, G.conj().T)
                assert np.all(G.diagonal().imag == 0)


@pytest.mark.parametrize("H,W,ap,step,P,Q", SHAPES[:8])
def test_strip_integer_exact(oracle_mod, H, W, ap, step, P, Q):
    img_np = wl.integer_valued((H, W), 60 + H, dtype="c64")
    img = torch.from_numpy(img_np).cuda()
    R = cov.apertures(img, ap, step, P, Q, norm="sum")
    torch.cuda.synchronize()
    got = R.cpu().numpy()
    nr, nc, sub = split(img_np, ap, step)
    for a in range(nr):
        for b in range(nc):
            S = oracle_mod.cov_window(sub(a, b).astype(np.complex128), P, Q, mean=False)
            assert np.array_equal(got[a * nc + b], S.astype(np.complex64)), (a, b)


def test_strip_agrees_with_the_batched_plan(oracle_mod):
    img_np = wl.complex_normal((95, 120), 91, dtype="c64")
    img = torch.from_numpy(img_np).cuda()
    R1 = cov.apertures(img, (25, 25), (10, 10), 10, 10)
    plan, R2 = cov.aperture_batch(img, (25, 25), (10, 10), 10, 10)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.upload(ws)
    plan.run(ws)
    torch.cuda.synchronize()
    cov.check_device_status(ws)
    a, b = R1.cpu().numpy(), R2.cpu().numpy()
    for k in range(a.shape[0]):
        assert rel_fro(a[k], b[k]) < 2 * F32_TOL


def test_strip_graph_capture_and_stream():
    img = torch.from_numpy(wl.complex_normal((75, 95), 92, dtype="c64")).cuda()
    s = torch.cuda.Stream()
    R0 = cov.apertures(img, (25, 25), (10, 10), 10, 10, stream=s)
    torch.cuda.synchronize()
    first = R0.cpu().numpy().copy()
    out = torch.full_like(R0, complex(np.nan, np.nan))
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        cov.apertures(img, (25, 25), (10, 10), 10, 10, out=out, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), first)  # same launch, same sums


def test_strip_full_image_sampled(oracle_mod):
    # 1015 x 1015 image, 100 x 100 apertures of 25 x 25 at stride 10, 10 x 10 window
    img_np = wl.complex_normal((1015, 1015), 77, "c64")
    img = torch.from_numpy(img_np).cuda()
    R = cov.apertures(img, (25, 25), (10, 10), 10, 10)
    torch.cuda.synchronize()
    assert R.shape == (10000, 100, 100)
    nr, nc, sub = split(img_np, (25, 25), (10, 10))
    rng = np.random.default_rng(3)
    picks = [(0, 0), (99, 99), (0, 99), (99, 0), (50, 3)] + [tuple(x) for x in rng.integers(0, 100, (15, 2))]
    for a, b in picks:
        want = oracle_mod.cov_window(sub(a, b).astype(np.complex128), 10, 10)
        assert rel_fro(R[a * nc + b].cpu().numpy(), want) < F32_TOL, (a, b)
