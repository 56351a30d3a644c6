"""The segmentation-quality metrics of §IV on hand-made cases (no GPU)."""
import numpy as np
import pytest

from paper_2003_00575_gb300 import quality


def test_hand_cases():
    # instances 1 (4 px) and 2 (2 px); pixel 6 is background
    gt = np.array([1, 1, 1, 1, 2, 2, 0])
    # a cluster holding instance 1 plus the background pixel, another holding instance 2
    lab = np.array([5, 5, 5, 5, 9, 9, 5])
    iou = quality.instance_ious(lab, gt, min_points=1)
    assert iou == {1: 4 / 5, 2: 1.0}
    # one cluster for both: instance 1 keeps it (4/6 > 2/6), instance 2 is not found
    lab = np.array([3, 3, 3, 3, 3, 3, -1])
    assert quality.instance_ious(lab, gt, min_points=1) == {1: 4 / 6, 2: 0.0}
    # instance 2 entirely unsegmented
    lab = np.array([0, 0, 0, 0, -1, -1, -1])
    assert quality.instance_ious(lab, gt, min_points=1) == {1: 1.0, 2: 0.0}
    # the size filter: only instance 1 has at least 3 points
    assert set(quality.instance_ious(lab, gt, min_points=3)) == {1}


def test_largest_overlap_and_ties():
    gt = np.array([1, 1, 1, 1, 1, 1])
    lab = np.array([7, 7, 8, 8, 8, -1])  # 8 overlaps more
    assert quality.instance_ious(lab, gt, 1) == {1: 3 / 6}
    lab = np.array([7, 7, 7, 8, 8, 8])   # a tie: the lower cluster id
    assert quality.instance_ious(lab, gt, 1) == {1: 3 / 6}


def test_scores_and_precision_bins():
    gt = np.repeat(np.arange(1, 5), 10)          # four instances of 10 px
    lab = gt.copy()
    lab[:1] = -1                                 # instance 1: IoU 0.9
    lab[10:15] = 99                              # instance 2: IoU 0.5 (5 of 10, cluster 5 px)
    lab[20:30] = 3                               # instance 3 merged into instance 4's cluster:
    lab[30:40] = 3                               # IoU 0.5 each, one kept (3), one not found
    s = quality.scores(lab, gt, min_points=10)
    assert s["instances"] == 4
    ious = sorted(quality.instance_ious(lab, gt, 10).values())
    assert ious == [0.0, 0.5, 0.5, 0.9]
    assert s["iou_mu"] == pytest.approx(np.mean(ious), abs=1e-4)
    assert s["p_50"] == 0.75 and s["p_75"] == 0.25 and s["p_95"] == 0.0
    assert s["p_mu"] == pytest.approx((0.75 + 0.25 * 8 + 0.0) / 10)


def test_perfect_and_pooled():
    g = np.random.default_rng(0)
    gt = g.integers(0, 6, 500)
    s = quality.scores(gt.copy(), gt, min_points=1)
    assert s["iou_mu"] == 1.0 and s["p_mu"] == 1.0
    pooled = quality.scores([gt, gt], [gt, gt], min_points=1)
    assert pooled["instances"] == 2 * s["instances"]
