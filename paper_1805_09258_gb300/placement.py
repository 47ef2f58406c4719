"""Adaptive record placement (Sec. 6): add records until every candidate point is covered.

Waves run from coarse to fine grid levels.  In wave `level` every cell of a 2^level grid
over the unit cube that still holds an uncovered pool candidate (whose own level is at
most `level`) gets one site -- the candidate with the smallest index (vrc_select_sites);
full records are computed at the sites (vrc_compute_records), the grid is rebuilt and
the candidates are queried (vrc_query_inscatter); covered candidates leave the pool
(vrc_update_coverage).  The waves end early once no candidate is left in the pool (site
selection reports the pool's size).  Candidates still uncovered after the finest wave get
a record each.  Coverage always uses the full records' radii, so the result honours the error
tolerance whatever picked the sites.

Plain placement starts every candidate at the coarsest level.  Learned placement first
predicts each candidate's radius from its coarse ray set (vrc_coarse_features,
vrc_mlp_predict) and lets it join only at the wave whose cell matches that radius
(vrc_levels_from_radius): regions of small radius skip the coarse waves, whose records
would cover almost nothing there.  A prediction made at the training tolerance is carried
to the placement's tolerance (R goes as eps^(1/5), Eq. radiusAniso3D), and it is kept only
where a record of the coarse ray set itself puts the error at the predicted radius within
the tolerance (vrc_mlp_fallback); elsewhere the candidate falls back to plain placement.

Batched learned placement places the sites of every predicted level in each wave: one
selection pass over all levels (vrc_select_sites_levels), one record launch, one grid
build and one coverage query per wave; the candidates a wave leaves uncovered move one
level finer (vrc_bump_levels) for the next wave.

One-shot learned placement selects the sites of every predicted level at once
(level by level on a copy of the pool, vrc_retire_level) and computes all their records
in one persistent launch, with one grid build and one coverage query; the few candidates
left uncovered then go through the plain waves at their predicted levels.

This module only sequences library calls; all work runs in libvrc's kernels.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import dataclasses
import math

from . import (MLP, Grid, Scene, alloc_records, bump_levels, coarse_features, compute_records, init_levels,
               levels_by_cell, levels_from_radius, mlp_fallback, query_inscatter, retire_level, select_sites,
               select_sites_levels, update_coverage,
               _torch)


_SIDE = {}


def _side_stream(torch, device):
    """One second stream per device, kept for the process (created once)."""
    key = torch.device(device).index
    if key not in _SIDE:
        _SIDE[key] = torch.cuda.Stream(device=device)
    return _SIDE[key]


@dataclass
class PlacementResult:
    n_records: int
    waves: list = field(default_factory=list)      # (level, sites) per wave
    seconds: float = 0.0
    records: dict = None
    grid: Grid = None
    uncovered_after_waves: int = 0
    predicted_sites: int = 0
    fallback_sites: int = 0


def place(scene: Scene, params, cand, start_level: int = 2, max_level: int = 7, mlp: MLP = None,
          coarse_params=None, cell_over_radius: float = 1.0, capacity: int = None, valid=None,
          base: PlacementResult = None, predict_level: int = 5, aniso: bool = False, eps_train: float = None,
          fallback: bool = True, one_shot: bool = False, batched: bool = False) -> PlacementResult:
    """Place records until every candidate point `cand` [n,3] (CUDA float32) is covered.

    valid [n] (int32, nullable): only nonzero entries are candidates.  base: an earlier
    placement whose records are kept (the new records are appended after them).
    aniso: records cover their ellipsoids (anisotropic cache points) instead of spheres.
    Learned placement (mlp given): eps_train is the tolerance the predictor was trained at
    (default params.eps); fallback applies the coarse-record check; one_shot places every
    predicted level's sites in one batched launch before the waves; batched runs every wave
    over all levels at once (uncovered candidates one level finer after each).
    """
    torch = _torch()
    n = cand.shape[0]
    t0 = time.perf_counter()
    prev = 0 if base is None else base.n_records
    cap = capacity or (prev + n)
    recs = alloc_records(cap, full=False, aniso=aniso)
    if prev:
        for k, v in base.records.items():
            recs[k][:prev].copy_(v)
    level = torch.empty((n,), dtype=torch.int32, device=cand.device)
    if valid is None:
        level.fill_(start_level)
    else:
        init_levels(valid, level, start_level)
    fine = min(8, max_level + 1)
    scratch = torch.empty((8 ** fine + 2 * n + n // 1024 + 3,), dtype=torch.int32, device=cand.device)
    site_idx = torch.empty((n,), dtype=torch.int32, device=cand.device)
    site_pts = torch.empty((n, 3), dtype=torch.float32, device=cand.device)
    res = PlacementResult(0)
    n_fallback = None
    if mlp is not None:
        # predict once per cell of a 2^predict_level grid (its smallest-index candidate)
        # and give every candidate of the cell that level
        m = select_sites(cand, level, predict_level, scratch, site_idx, site_pts)
        if m:
            pts = site_pts[:m].contiguous()
            main = torch.cuda.current_stream()
            rc = None
            if fallback:
                # the coarse ray set's own record at the placement's tolerance, on a second
                # stream while the features and the prediction run on this one (the two read
                # only the scene and the sites)
                side = _side_stream(torch, cand.device)
                side.wait_stream(main)
                cp = dataclasses.replace(params, n_bands=coarse_params.n_bands, n_bins=coarse_params.n_bins,
                                         seed=coarse_params.seed, rec_base=0, parts=0)
                with torch.cuda.stream(side):
                    rc = compute_records(scene, pts, cp, full=False)["radius"]
                pts.record_stream(side)
            feat = coarse_features(scene, pts, coarse_params, bf16=True)     # read by TMA in the forward pass
            logr = mlp.predict(feat)
            offset = 0.2 * math.log(params.eps / (eps_train or params.eps))
            if rc is not None:
                main.wait_stream(side)
                rc.record_stream(main)
            logr, n_fallback = mlp_fallback(logr, offset, rc, logr_fallback=10.0)
            res.predicted_sites = m
            rep = torch.empty((n,), dtype=torch.int32, device=cand.device)
            levels_by_cell(cand, predict_level, scratch, site_idx, logr, m, cell_over_radius, start_level, max_level,
                           rep, level)
    count = torch.empty((n,), dtype=torch.int32, device=cand.device)
    rgb = torch.empty((n, 3), dtype=torch.float32, device=cand.device)
    total = prev
    grid = base.grid if base is not None else None
    base_grid = grid                      # the caller's grid is never rebuilt in place
    if grid is not None:
        query_inscatter(grid, cand, rgb, count)
        update_coverage(count, level)

    def add_records(pts, m):
        nonlocal total, grid
        if total + m > cap:
            raise RuntimeError("placement capacity exceeded")
        out = {k: v[total:total + m] for k, v in recs.items()}
        compute_records(scene, pts[:m].contiguous(), params, out=out)
        total += m
        view = {k: v[:total] for k, v in recs.items()}
        if grid is not None and grid is not base_grid and grid.aniso == aniso:
            grid.rebuild(view, n=total)
        else:
            grid = Grid(view, n=total, aniso=aniso)
        query_inscatter(grid, cand, rgb, count)
        update_coverage(count, level)

    if one_shot and mlp is not None:
        # every predicted level's sites at once: level by level on a copy of the pool, each
        # level's candidates retired after its selection, then one batched record launch
        pool = level.clone()
        batch = torch.empty((n, 3), dtype=torch.float32, device=cand.device)
        got = 0
        for lv in range(start_level, max_level + 1):
            m = select_sites(cand, pool, lv, scratch, site_idx, site_pts)
            if m:
                batch[got:got + m].copy_(site_pts[:m])
                got += m
            retire_level(pool, lv)
        res.waves.append(("one-shot", got))
        if got:
            add_records(batch, got)
    in_pool = n
    if batched and mlp is not None:
        # every level's sites in one wave (one selection pass, one record launch, one grid
        # build and coverage query); the candidates a wave leaves uncovered move one level
        # finer for the next; those past max_level go to the fine fill below
        while True:
            m, in_pool = select_sites_levels(cand, level, start_level, max_level, scratch, site_idx, site_pts)
            if in_pool == 0 or m == 0:
                break
            res.waves.append(("levels", m))
            add_records(site_pts, m)
            bump_levels(level, fine)
    else:
        for lv in range(start_level, max_level + 1):
            m, in_pool = select_sites(cand, level, lv, scratch, site_idx, site_pts, with_pool=True)
            if in_pool == 0:
                break                         # every candidate is covered: the finer waves are empty
            res.waves.append((lv, m))
            if m:
                add_records(site_pts, m)
    # candidates still uncovered get sites on the finest grid until none is left (each
    # wave covers at least its own sites, so this ends)
    left = 0 if in_pool == 0 else select_sites(cand, level, fine, scratch, site_idx, site_pts)
    res.uncovered_after_waves = left
    while left:
        add_records(site_pts, left)
        res.waves.append((fine, left))
        left = select_sites(cand, level, fine, scratch, site_idx, site_pts)
    torch.cuda.synchronize()
    res.seconds = time.perf_counter() - t0
    if n_fallback is not None:
        res.fallback_sites = int(n_fallback.item())
    res.n_records = total
    res.records = {k: v[:total] for k, v in recs.items()}
    res.grid = grid
    return res
