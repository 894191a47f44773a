"""Every aperture of one image through one batched launch, read in place
(no copies), against the oracle on each extracted aperture."""
import numpy as np
import pytest
import torch

import cov_workloads as wl
import paper_1303_2285_gb300 as cov

pytestmark = pytest.mark.gpu

from gpu_util import rel_fro  # noqa: E402


@pytest.mark.parametrize("H,W,ap,step,P,Q", [(64, 80, (25, 25), (10, 10), 10, 10),
                                             (47, 51, (20, 17), (9, 5), 4, 3),
                                             (40, 40, (40, 40), (1, 1), 16, 16)])
def test_apertures_match_oracle(oracle_mod, H, W, ap, step, P, Q):
    img_np = wl.complex_normal((H, W + 7), 31 + H, dtype="c64")  # ld = W + 7
    img = torch.from_numpy(img_np).cuda()[:, :W]
    plan, R = cov.aperture_batch(img, ap, step, P, Q)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.upload(ws)
    plan.run(ws)
    torch.cuda.synchronize()
    cov.check_device_status(ws)
    got = R.cpu().numpy()
    nr, nc = (H - ap[0]) // step[0] + 1, (W - ap[1]) // step[1] + 1
    assert got.shape[0] == nr * nc
    for a in range(nr):
        for b in range(nc):
            sub = img_np[a * step[0]:a * step[0] + ap[0], b * step[1]:b * step[1] + ap[1]]
            want = oracle_mod.cov_window(sub.astype(np.complex128), P, Q)
            assert rel_fro(got[a * nc + b], want) < 1e-5
