"""Comparison helpers for the GPU parity tests (no model arithmetic)."""
import numpy as np

GRAZE = 2e-4  # grazing band, in link lengths


def oracle_poses(orc, ost, i):
    th = orc.theta_of(ost, i)
    px, py, psi = orc.poses(i, th, ost["l"][i])
    return th, px, py, psi


def pose_error(batch, st, orc, ost, i):
    """Max position error (m) over link start points and tip, and max heading error (rad)."""
    th, px, py, psi = oracle_poses(orc, ost, i)
    pose = batch.pose_of(st, i)
    if pose.shape[0] != th.size:
        return np.inf, np.inf
    e = max(np.max(np.abs(pose[:, 0] - px[:-1]), initial=0.0), np.max(np.abs(pose[:, 1] - py[:-1]), initial=0.0),
            abs(st["tip"][i, 0] - px[-1]), abs(st["tip"][i, 1] - py[-1]))
    eh = np.max(np.abs(pose[:, 2] - psi), initial=0.0)
    return float(e), float(eh)


def contact_sets(counts, pairs, orc, ost, i, l_seg):
    """(gpu_set, oracle_set, grazing_set) of (link, obstacle) pairs."""
    gpu = {tuple(p) for p in pairs[i, : counts[i]]}
    th = orc.theta_of(ost, i)
    gap = orc.gaps(i, th, ost["l"][i])
    band = GRAZE * l_seg
    orc_set = {(int(a), int(b)) for a, b in zip(*np.nonzero(gap < 0))}
    graze = {(int(a), int(b)) for a, b in zip(*np.nonzero(np.abs(gap) <= band))}
    return gpu, orc_set, graze


def contacts_match(gpu, orc_set, graze):
    return (gpu - graze) == (orc_set - graze)
