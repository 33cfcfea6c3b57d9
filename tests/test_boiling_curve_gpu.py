"""Fig. 11 at the paper's scale (Section 4.4, qualitative): 400 x 600 pools on a
25-row heater with three nucleation sites (minima 0, -0.3, -0.6), advanced
together by the batched step for 60,000 steps; the wall heat flux and the wall
vapour coverage are averaged over the second half.  The curve must show the
paper's regimes in order: no vapour at the wall below the onset of nucleate
boiling (Ja <= 0.08), boiling from Ja = 0.11, a flux that rises with Ja to a
maximum between Ja = 0.166 and 0.21 (the paper's critical heat flux is near
0.186), and a drop past it as a vapour film covers most of the wall.  The GPU
step behind it is pinned to the FP64 oracle by the parity tests; this test
compares with the paper's figure, not with the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1812_10375_gb300 import build
    build.build()


def test_paper_scale_boiling_curve_shape():
    from paper_1812_10375_gb300 import sweep
    ja = [0.05, 0.08, 0.11, 0.13, 0.15, 0.166, 0.176, 0.186, 0.197, 0.21, 0.22, 0.25]
    rows, seconds = sweep.paper_curve(ja, 60000)
    q = np.array([r["q"] for r in rows])
    cov = np.array([r["coverage"] for r in rows])
    for r in rows:
        print(f"Ja {r['Ja']:.3f}: q {r['q']:.3e} h {r['h']:.4f} coverage {r['coverage']:.3f} regime {r['regime']}")
    print(f"{len(rows)} points x 60000 steps of 400 x 600 in {seconds:.1f} s")
    ja = np.array(ja)
    assert np.all(cov[ja <= 0.08] < 0.005)            # below the onset: no vapour at the wall
    assert np.all(cov[(ja >= 0.13) & (ja <= 0.21)] > 0.02)
    k = int(np.argmax(q))
    assert 0.166 <= ja[k] <= 0.21                     # maximum flux where the paper puts it
    assert np.all(np.diff(q[: k + 1])[2:] > 0)        # rising from the onset to the maximum
    assert q[-1] < 0.7 * q[k]                         # past the maximum the flux drops
    assert cov[ja >= 0.22].max() > 0.5                # as a vapour film covers the wall
