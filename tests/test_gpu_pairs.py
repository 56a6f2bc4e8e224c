"""The sweep with each phase pair's patch distances computed once (the
symmetric reuse of Sec. 2.4, tnlm_gauss_jacobi_pairs) against the FP64
oracle's sweep and against the direct sweep."""
import numpy as np
import pytest
import torch

import paper_1201_2450_gb300 as tnlm
from paper_1201_2450_gb300 import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("shape, d, M, clip", [((3, 9, 13, 19), 1, 3, 1),    # ragged against every tile
                                               ((3, 7, 10, 11), 2, 3, 0),
                                               ((2, 8, 12, 20), 2, 1, 1),    # N_p = 2: both directions, one pair
                                               ((5, 17, 23, 35), 1, 2, 0),
                                               ((4, 12, 30, 29), 2, 2, 1)])
def test_pair_sweep_matches_oracle_and_direct_sweep(ora, shape, d, M, clip):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    tnlm.build()
    a = synth.smooth_volume(shape, 700) + synth.normal(shape, 701, 0.003)
    v = synth.smooth_volume(shape, 702)
    g = synth.smooth_volume(shape, 703)
    h = 0.02
    A, V, G = (torch.from_numpy(t).cuda() for t in (a, v, g))
    out = tnlm.tnlm_gauss_jacobi_pairs(A, V, G, d, M, h, 0.9, clip)
    ref = ora.gj_sweep(a, v, g, d, M, h, 0.9, clip)
    direct = tnlm.tnlm_gauss_jacobi(A, V, G, d, M, h, 0.9, clip)
    err = rel_l2(out.cpu().numpy(), ref)
    print(f"pair sweep {shape} d={d} M={M}: rel-L2 vs FP64 {err:.2e}, vs direct "
          f"{rel_l2(out.cpu().numpy(), direct.cpu().numpy()):.2e}")
    assert err <= RTOL
    assert rel_l2(out.cpu().numpy(), direct.cpu().numpy()) <= 1e-6


def test_pair_sweep_enhancement_structure(ora):
    """TNLM-E's structure (d = 2, M = 3, h = 0.04, streaked input) for three
    sweeps composed from pair sweeps, against the oracle's TNLM-E."""
    cfg = synth.EnhanceConfig("t", 4, (26, 22, 14), 1.0, 0.002, 0.003, 36, 2, 3, 0.04, 1.0, 3, 221)
    g, _ = synth.enhance_input(cfg)
    G = g.cuda()
    f = G
    for _ in range(3):
        f = tnlm.tnlm_gauss_jacobi_pairs(f, f, G, 2, 3, 0.04, 1.0, 0)
    ref = ora.enhance(g.numpy(), 2, 3, 0.04, 1.0, 3)
    assert rel_l2(f.cpu().numpy(), ref) <= RTOL
