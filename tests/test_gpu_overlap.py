"""rsf_overlap (Dice and Jaccard, Sec. 5.3) against the oracle's counts, on
device and host buffers, and a segmentation of the light-sheet workload
scored against the generator's ground truth."""
import numpy as np
import pytest

import oracle
from paper_2404_02813_gb300 import rsf, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    c = rsf.Context(0)
    yield c
    c.close()


def test_counts_match_oracle(ctx):
    rng = np.random.default_rng(12)
    phi = rng.normal(0, 1, size=(37, 41, 53)).astype(np.float32)
    phi[0, 0, :5] = 0.0  # phi = 0 is outside
    truth = rng.random(phi.shape) < 0.3
    want = oracle.overlap_counts(phi, truth)
    for p, t in [(torch.from_numpy(phi).cuda(), torch.from_numpy(truth).cuda()), (phi, truth)]:
        got = ctx.overlap(p, t)
        assert (got["segmented"], got["truth"], got["both"]) == want
        d, j = oracle.dice_jaccard(want)
        assert abs(got["dice"] - d) < 1e-12 and abs(got["jaccard"] - j) < 1e-12


def test_lightsheet_segmentation_score(ctx):
    vol, truth = synth.lightsheet_volume_u16((64, 96, 128), truth=True)
    phi0 = synth.mean_rule_phi0(vol)
    p = dict(sigma=3.0, eps=1.0, lambda1=1.0, lambda2=2.0, nu=0.004 * 4300.0 ** 2, mu=1.0, dt=0.1)
    out = ctx.evolve(torch.from_numpy(vol).cuda(), torch.from_numpy(phi0).cuda(), p, 200)
    got = ctx.overlap(out, torch.from_numpy(truth).cuda())
    want = oracle.overlap_counts(out.cpu().numpy(), truth)
    assert (got["segmented"], got["truth"], got["both"]) == want
    print(f"light-sheet 128x96x64 after 200 iterations: Dice {got['dice']:.4f}, Jaccard {got['jaccard']:.4f}")
    assert 0.0 <= got["dice"] <= 1.0
