"""The GPU parity cases reach every staging path of the fused kernel's inputs.

Per 128-sample tile the row setup reduces the rows' opacity-table rows and source cells and
the fused kernel stages, for each stage of 16 spectral points, either a small box (a tile whose
rows span one or two table rows / stay in one row of cube cells), the full box (up to 8 table
rows / 11 x 3 cube cells with the bilinear neighbours), or nothing (the rows read global memory).
This host test recomputes the tiles' extents from the oracle's geometry (Sect. 2.4, Eqs. 9-10) for
the parity cases and checks that, between them, every path is taken, so a change of the
scenarios cannot quietly leave one untested.
"""
import importlib.util
import os

import numpy as np

from oracle import gateau_oracle as O
from paper_2604_23305_b300 import workloads as W

TILE = 128
TAU_ROWS, TAU_ROWS_SMALL = 8, 2          # opacity rows of the full and the small box
CUBE_AZ, CUBE_EL, CUBE_EL_SMALL = 12, 4, 2


def _edge_cases():
    path = os.path.join(os.path.dirname(__file__), "test_gpu_parity.py")
    spec = importlib.util.spec_from_file_location("gpu_parity_cases", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.EDGE


def tile_paths(sc, t0, nt):
    """Set of (opacity path, cube path) over the tiles of rows t0 .. t0 + nt - 1 of every spaxel."""
    src, atm = sc["source"], sc["atmosphere"]
    n_az, n_el = src["cube"].shape[0], src["cube"].shape[1]
    n_pwv = np.asarray(atm["table"]).shape[0]
    n = np.arange(t0, t0 + nt)
    paths = set()
    for i in range(len(sc["pix_offsets"])):
        _, az, el, pwv = O.row_geometry(sc, n, np.full(nt, i))
        u = np.clip((pwv - atm["pwv_min"]) / atm["dpwv"], 0, n_pwv - 1)
        j = np.minimum(np.floor(u).astype(int), n_pwv - 2)
        su, sv = (az - src["az0"]) / src["daz"], (el - src["el0"]) / src["del"]
        inside = (su >= 0) & (su <= n_az - 1) & (sv >= 0) & (sv <= n_el - 1)
        ia = np.minimum(np.floor(su).astype(int), n_az - 2)
        ie = np.minimum(np.floor(sv).astype(int), n_el - 2)
        # tiles are aligned to the run's first sample, as in the row setup
        for b in range(0, nt, TILE):
            span = j[b:b + TILE].max() - j[b:b + TILE].min()
            tau = "small" if span <= TAU_ROWS_SMALL - 1 else ("full" if span <= TAU_ROWS - 1 else "global")
            m = inside[b:b + TILE]
            if not m.any():
                cube = "none"
            else:
                a, e = ia[b:b + TILE][m], ie[b:b + TILE][m]
                fits = a.max() + 1 - a.min() <= CUBE_AZ - 1 and e.max() + 1 - e.min() <= CUBE_EL - 1
                small = e.max() + 1 - e.min() <= CUBE_EL_SMALL - 1
                cube = ("small" if small else "full") if fits else "global"
            paths.add((tau, cube))
    return paths


def test_parity_cases_reach_every_staging_path():
    taken = set()
    for name, t0, nt, mut in _edge_cases().values():
        sc = W.scenario(name, nt_total=max(t0 + nt, 1))
        if mut:
            mut(sc)
        taken |= tile_paths(sc, t0, nt)
    # the headline workload's tiles take both small boxes
    taken |= tile_paths(W.scenario("ifu25", nt_total=300), 0, 300)
    assert {t for t, _ in taken} >= {"small", "full", "global"}, taken
    assert {c for _, c in taken} >= {"small", "full", "global", "none"}, taken
