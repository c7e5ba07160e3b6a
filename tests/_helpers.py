"""Shared test utilities (no response arithmetic beyond what each test states)."""
import numpy as np

import synth

C = synth.C_LIGHT
LINKS = [(1, 2), (2, 3), (3, 1), (1, 3), (3, 2), (2, 1)]   # (receiver, emitter)
LINK_INDEX = {f"{r}{s}": l for l, (r, s) in enumerate(LINKS)}


def k_vector(lam, beta):
    """Propagation direction k = -e_r of the paper's SSB frame."""
    return -np.array([np.cos(beta) * np.cos(lam), np.cos(beta) * np.sin(lam), np.sin(beta)])


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def relabel_positions(pos, perm):
    """pos'[i] = pos[perm[i]] for 0-based spacecraft indices."""
    return np.stack([pos[perm[i]] for i in range(3)])


def constant_orbit_from(pos3x3, delays6, t_start, t_end):
    tk = synth.knot_grid(t_start, t_end, 1e5)
    pos = np.repeat(np.asarray(pos3x3, dtype=float)[:, :, None], len(tk), axis=2)
    dl = np.repeat(np.asarray(delays6, dtype=float)[:, None], len(tk), axis=1)
    return tk, pos, dl
