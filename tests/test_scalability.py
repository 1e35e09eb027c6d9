"""Scalability study (Fig. 3f/g): the synthetic disk images, and on the GPU
the timing helpers and the feature-group split."""
import numpy as np
import pytest
import scipy.ndimage as ndi

from paper_2603_12016_gb300 import workloads as W


@pytest.mark.parametrize("px,n", [(100, 50), (5000, 9), (20000, 4)])
def test_disk_workload_sizes_and_separation(px, n):
    w = W.scalability_2d(px, n, seed=3)
    labels, counts = np.unique(w.mask[w.mask > 0], return_counts=True)
    assert labels.size == n and w.meta["n_roi"] == n
    assert np.all(np.abs(counts - px) <= 0.06 * px + 4), counts
    # no two disks touch: every 8-connected component is one whole label
    comp, ncomp = ndi.label(w.mask > 0, structure=np.ones((3, 3)))
    assert ncomp == n


@pytest.mark.gpu
def test_timing_helpers_and_groups():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12016_gb300 import build
    from paper_2603_12016_gb300 import scalability as S

    build.build()
    w = W.scalability_2d(20000, 16, seed=5)
    dev = S.time_device(w, steps=5)
    e2e = S.time_end_to_end(w, steps=3)
    assert 0 < dev and e2e["h2d_bytes"] == w.image.nbytes + w.mask.nbytes
    g = S.group_costs(w, steps=5)
    assert set(g) == {"intensity", "moments", "texture", "all"} and all(v > 0 for v in g.values())
    # every group alone costs no more than the whole feature set (10% timing
    # slack; the texture group is most of the set on ROIs this large)
    assert max(g["intensity"], g["moments"], g["texture"]) <= 1.1 * g["all"]


def test_groups_cover_every_feature_once():
    """The groups split the library's feature registry: every id in exactly
    one group (checked against the C ABI's name lookup, no GPU)."""
    from paper_2603_12016_gb300 import build
    from paper_2603_12016_gb300 import scalability as S

    build.build()
    from paper_2603_12016_gb300 import nyx

    ids = [nyx.feature_id(n) for g in S.GROUPS.values() for n in g]
    assert min(ids) >= 0
    # the registry holds ids 0..138; the last one is the final GLSZM feature
    assert sorted(ids) == list(range(139)) and nyx.feature_id("GLSZM_ZSM") == 138
    assert set(S.NGTDM + S.GLDM + S.GLRLM + S.GLSZM) <= set(S.GROUPS["texture"])
