"""Whole sweeps on both paths against the oracle, with the error stated per frequency set
(needs a CUDA GPU; slow: the oracle's sweep takes minutes at 512^2).

For breast256 (4 sets of 3 frequencies) and breast512, the benchmarked workload (5 sets
of 4 frequencies), the oracle's data p_obs (its ray-Born forward model plus the seeded
1 % noise) feed both sides.  Per set j:
  * one rb_hf_update started from the oracle's own sound speed before set j, against
    oracle.update.hf_update from the same c: dc relative L2, the step scale, ||dc|| and
    the data counts;
  * an independent GPU sweep from c_init, compared with the oracle's sweep after every
    set: the RMS of the c difference over the support (bar 0.05 m/s after the last set,
    the bound the reconstruction is held to).
The per-set numbers are printed (pytest -s) on the FP32 and the BF16 x3 path.

Bars per set: dc, the step scale and ||dc|| within 1e-3 where no ray of the set's
medium crosses a caustic.  Once the updated medium folds some fans (the later sets at
512^2), the amplitude sqrt(c / (8 pi w J)) of the entries next to a caustic, where the
tube width J = |Q| passes through zero, is ill-conditioned: Q agrees to ~1e-6 of its
scale between FP32 and FP64, which is a percent of J there.  Those few entries carry
most of the difference (at 512^2, set 3: the largest 1 % of pixels hold 77 % of its
norm, 3.5e-3 relative), so such sets are held to 2e-2 (1e-2 on the step scale and
||dc||).

The independent sweeps are held to the 0.05 m/s bound while the media they pass
through leave at most 0.1 % of the rays past a caustic (the whole sweep at 256^2, the
first three sets at 512^2).  Beyond that the map from c to the update is not
continuous: where fans fold, a first-arrival winner flips between triangles of
different sheets of the fan under any perturbation of c, and its Green's function
changes by O(1) there.  A 0.001 m/s difference between the two sweeps after set 2 at
512^2 grows to 0.12 m/s after set 3 (the same update from the same c differs by only
0.02 m/s) and 1.1 m/s after set 4, on either path; those values are reported, not
held to the bound.
"""
import math

import numpy as np
import pytest

import rbgen
from oracle import geometry as ogeom
from oracle import rays as orays
from oracle import update as oupd
from oracle.rays import VK

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from paper_2511_16633_gb300 import rb  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rb.load()
    return torch.device("cuda:0")


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


_REFS = {}


def _oracle_sweep(name):
    """The oracle's sweep with every set's starting c and result kept."""
    if name not in _REFS:
        cfg = rbgen.config_by_name(name)
        inp = rbgen.make_inputs(cfg)
        g = ogeom.from_config(cfg)
        p_obs = oupd.synth_data(g, inp.c_init, inp.c_true, inp.alpha0, cfg.freqs_hz, inp.noise_re, inp.noise_im)
        c = np.asarray(inp.c_init, dtype=np.float64)
        sets = []
        for s in cfg.sets:
            fs = [cfg.freqs_hz[i] for i in s]
            r = oupd.hf_update(g, c, inp.alpha0, fs, p_obs[list(s)])
            E, _, _ = orays.trace_endpoints(g, c, inp.alpha0)
            sets.append(dict(c0=c.copy(), freqs=fs, idx=list(s), dc=r.dc, alpha=r.alpha, norm=r.dc_norm,
                             kept=r.n_kept, zeroed=r.n_zeroed, c1=r.c_new.copy(),
                             caustic_rays=int(np.sum(E[..., VK] > 0))))
            c = r.c_new
        _REFS[name] = (cfg, inp, g, p_obs, sets)
    return _REFS[name]


@pytest.mark.parametrize("name", ["breast256", "breast512"])
@pytest.mark.parametrize("prec", [rb.RB_PREC_FP32, rb.RB_PREC_BF16X3], ids=["fp32", "bf16x3"])
def test_sweep_per_set_against_the_oracle(dev, name, prec):
    cfg, inp, g, p_obs, sets = _oracle_sweep(name)
    geom = rb.geometry_from_config(cfg)
    sup = ogeom.support_mask(g)
    a0 = torch.as_tensor(np.asarray(inp.alpha0, np.float32), device=dev)
    p = torch.as_tensor(p_obs.astype(np.complex64), device=dev)
    nmax = max(len(s["freqs"]) for s in sets)
    ws = rb.workspace(geom, nmax, prec, dev)
    dc = torch.empty((g.ny, g.nx), dtype=torch.float32, device=dev)
    diag = torch.zeros(48, dtype=torch.uint8, device=dev)
    c_sweep = torch.as_tensor(np.asarray(inp.c_init, np.float32), device=dev).clone()
    dc_sw = torch.empty_like(dc)
    diag_sw = torch.zeros_like(diag)
    lo = lambda s: s["idx"][0]
    hi = lambda s: s["idx"][-1] + 1
    rows = []
    for j, s in enumerate(sets):
        # the set's update from the oracle's own c before it
        c = torch.as_tensor(s["c0"].astype(np.float32), device=dev)
        rb.rb_hf_update(geom, c, a0, s["freqs"], p[lo(s):hi(s)], ws, prec=prec, dc_out=dc, diag_out=diag)
        # the independent sweep's set j
        rb.rb_hf_update(geom, c_sweep, a0, s["freqs"], p[lo(s):hi(s)], ws, prec=prec, dc_out=dc_sw,
                        diag_out=diag_sw)
        torch.cuda.synchronize()
        d = rb.decode_diag(diag)
        e = rel_l2(dc.cpu().numpy(), s["dc"])
        crms = float(np.sqrt(np.mean((c_sweep.cpu().numpy().astype(np.float64) - s["c1"])[sup] ** 2)))
        assert d["lost_rays"] == 0 and d["tc_timeouts"] == 0 and rb.decode_diag(diag_sw)["tc_timeouts"] == 0
        assert d["zeroed"] == math.floor(0.01 * d["kept"])
        rows.append((j, e, d["alpha"] / s["alpha"] - 1.0, d["dc_norm"] / s["norm"] - 1.0, d["kept"] - s["kept"], crms,
                     s["caustic_rays"]))
    print(f"\n{name} {'fp32' if prec == rb.RB_PREC_FP32 else 'bf16x3'}: set, dc rel L2, alpha rel, ||dc|| rel, "
          f"kept diff, sweep c RMS diff [m/s], rays past a caustic")
    for r in rows:
        print(f"  {r[0]}  {r[1]:.3g}  {r[2]:+.2g}  {r[3]:+.2g}  {r[4]:+d}  {r[5]:.3g}  {r[6]}")
    n_rays = g.n_elem * g.n_rays
    smooth = True     # every medium so far leaves at most 0.1 % of the rays past a caustic
    for (j, e, ra, rn, dk, crms, ncau) in rows:
        bar, bar_s = (1e-3, 1e-3) if ncau == 0 else (2e-2, 1e-2)
        assert e <= bar, (j, e, ncau)
        assert abs(ra) <= bar_s and abs(rn) <= bar_s, (j, ra, rn)
        assert abs(dk) <= 1e-3 * sets[j]["kept"]
        smooth = smooth and ncau <= 1e-3 * n_rays
        if smooth:
            assert crms <= 0.05, (j, crms)
    if name == "breast256":
        assert smooth     # the whole sweep is held to the bound
