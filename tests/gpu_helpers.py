"""Shared helpers of the GPU parity tests: run the CUDA path, compare with the oracle.

The tolerances are those the method's acceptance criteria state: radiance within
1e-4 relative, gradient and Hessian within 1e-3 relative to their norms.  On top of
the relative tolerance, each record may differ by its decision-sensitivity budget,
computed by the oracle: the largest change that flipping its near-tie discrete
decisions (a shadow or primary ray passing within 1e-6 of a triangle edge, a shell
vertex within float rounding of its clamp, tied furthest vertices) could make.  A
record with no near-tie decision has a zero budget and is held to the bare tolerance.
"""
import numpy as np

TOL_L = 1e-4
TOL_D = 1e-3


def hess_fro(h6):
    h6 = np.asarray(h6, np.float64)
    return np.sqrt(h6[..., 0] ** 2 + h6[..., 3] ** 2 + h6[..., 5] ** 2 +
                   2.0 * (h6[..., 1] ** 2 + h6[..., 2] ** 2 + h6[..., 4] ** 2))


def to_np(out):
    return {k: v.detach().cpu().numpy() for k, v in out.items()}


def compare_records(gpu, ref, idx=None, parts=("", "_ss", "_ms")):
    """Check GPU records (dict of numpy arrays, rows idx) against oracle records (all rows).

    Returns a dict of statistics; raises AssertionError listing the failing records.
    """
    n = ref["L"].shape[0]
    idx = np.arange(n) if idx is None else np.asarray(idx)
    fails = []
    stats = dict(n=n, zero_budget=0, worst_L=0.0, worst_g=0.0, worst_H=0.0)
    for r in range(n):
        i = idx[r]
        zb = ref["bud_L"][r].max() == 0 and ref["bud_grad"][r].max() == 0 and ref["bud_hess"][r].max() == 0
        stats["zero_budget"] += int(zb)
        for part in parts:
            Lg, Lo = gpu["L" + part][i].astype(np.float64), ref["L" + part][r]
            errL = np.abs(Lg - Lo)
            tolL = TOL_L * np.abs(Lo) + ref["bud_L"][r] + 1e-12
            if np.any(errL > tolL):
                fails.append((int(i), "L" + part, errL.tolist(), tolL.tolist()))
            stats["worst_L"] = max(stats["worst_L"], float(np.max(errL / tolL)))
            gg = gpu["grad" + part][i].reshape(3, 3).astype(np.float64)
            go = ref["grad" + part][r].reshape(3, 3)
            hg = gpu["hess" + part][i].reshape(3, 6).astype(np.float64)
            ho = ref["hess" + part][r].reshape(3, 6)
            for c in range(3):
                eg = np.linalg.norm(gg[c] - go[c])
                tg = TOL_D * np.linalg.norm(go[c]) + ref["bud_grad"][r, c] + 1e-12
                eh = hess_fro(hg[c] - ho[c])
                th = TOL_D * hess_fro(ho[c]) + ref["bud_hess"][r, c] + 1e-12
                if eg > tg:
                    fails.append((int(i), f"grad{part}[{c}]", eg, tg))
                if eh > th:
                    fails.append((int(i), f"hess{part}[{c}]", eh, th))
                stats["worst_g"] = max(stats["worst_g"], eg / tg)
                stats["worst_H"] = max(stats["worst_H"], eh / th)
    assert not fails, f"{len(fails)} mismatches, first: {fails[:6]}"
    return stats


def compare_radius(gpu, ref, idx=None):
    """Radius R = (15 L eps / (4 pi |lambda|))^(1/5): its relative error is a fifth of the
    relative errors of L_Y and |lambda| (Weyl: |d lambda| <= ||dH||_F)."""
    n = ref["L"].shape[0]
    idx = np.arange(n) if idx is None else np.asarray(idx)
    Y = np.array([0.2126, 0.7152, 0.0722])
    for r in range(n):
        i = idx[r]
        Ro, Rg = ref["radius"][r], float(gpu["radius"][i])
        LY = float(ref["L_Y"][r])
        lam = float(ref["lam_max"][r])
        tLY = TOL_L * abs(LY) + float(Y @ ref["bud_L"][r])
        hy = (Y[:, None] * ref["hess"][r].reshape(3, 6)).sum(0)
        tH = TOL_D * hess_fro(hy) + float(Y @ ref["bud_hess"][r])
        rel = 0.2 * (tLY / max(abs(LY), 1e-30) + tH / max(lam, 1e-30)) + 1e-5
        st_o, st_g = int(ref["status"][r]), int(gpu["status"][i])
        clamped = st_o & 6 or st_g & 6
        if clamped:
            # both clamped to the same bound, or within tolerance of it
            assert abs(Rg - Ro) <= rel * Ro * 1.5 + 1e-7, (int(i), Rg, Ro, st_g, st_o)
        else:
            assert abs(Rg - Ro) <= rel * Ro, (int(i), Rg, Ro, rel)
        assert (st_o & 1) == (st_g & 1), (int(i), st_g, st_o)


def oracle_replayed(O, oscene, params, pos, g, rec_ids=None, n_bands=None, idx=None, track_margins=0):
    """The oracle on the GPU's own discrete decisions (replay mode): its primary hit ids,
    its FP32 ray ends (which decide the shell clamps and furthest vertices) and its
    visibility bits, from a launch with debug_hits (parts = 0).  The records are then
    computed in FP64 on the same decisions and compared with the bare tolerances; every
    replayed decision must be a near tie for the oracle (n_unexplained == 0)."""
    sel = slice(None) if idx is None else np.asarray(idx)
    ref = O.records(oscene, params, pos, rec_ids=rec_ids, n_bands=n_bands, track_margins=track_margins,
                    replay_hits=g["hit_prim"][sel], replay_t=g["hit_t"][sel], replay_lit=g["dbg_lit"][sel])
    bad = np.flatnonzero(ref["n_unexplained"] > 0)
    assert bad.size == 0, f"{bad.size} records with decisions that are not near ties, first {bad[:8]}"
    return ref
