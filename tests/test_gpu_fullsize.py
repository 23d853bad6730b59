"""Full-size parity: the headline workload (3-D Potts 128^3, L = 8, 64 chains)
in the launch configuration bench.py times, checked on sampled sites.

The oracle cannot sweep 134 M site updates, so it sweeps a compact sub-model:
the sampled sites, their incident edges and the neighbours at the far ends,
with the full model's edge slots and site ids as RNG indices.  A sampled
site's primal field only involves its incident edges, so its label draw is
exactly the full model's (neighbours' fields are incomplete and not compared).
"""
import numpy as np
import pytest

from oracle import decompose as dc, sampler
from paper_1611_06684_gb300 import workloads as wl
from gpu_helpers import BOUNDARY_EPS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_06684_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def headline():
    return wl.potts_grid3d(128, L=8, seed=0)


def _sub_model(model, sites):
    """Compact model of the sampled sites' incident edges; returns it with the
    global ids of its sites and edges."""
    inc = np.isin(model.src, sites) | np.isin(model.dst, sites)
    eids = np.nonzero(inc)[0]
    local = np.unique(np.concatenate([sites, model.src[eids], model.dst[eids]]))
    sub = wl.Model(n_vars=len(local), n_labels=model.n_labels, unary=model.unary[local],
                   src=np.searchsorted(local, model.src[eids]).astype(np.int32),
                   dst=np.searchsorted(local, model.dst[eids]).astype(np.int32),
                   pair=model.pair[eids], name="sub")
    return sub, local, eids


@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_headline_size_sampled_sites_match_oracle(headline, mode):
    from paper_1611_06684_gb300 import mrf as M
    model = headline
    C, seed = 64, 0
    h = M.MRF(model.n_vars, model.n_labels, C, seed=seed, kernel_timing=True, grid=model.grid)
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    md = M.MODE_PLAIN if mode == "plain" else M.MODE_FUSED
    h.sweep(3, md)
    t = h.info().sweep_index
    x0 = h.get_labels()
    h.sweep(1, md)
    x1 = h.get_labels()
    h.close()
    rng = np.random.default_rng(5)
    sites = np.sort(rng.choice(model.n_vars, size=600, replace=False))
    sub, local, eids = _sub_model(model, sites)
    dec = dc.decompose(sub)
    ref = sampler.sweep(dec, x0[:, local].astype(np.int64), t, seed, edge_ids=eids, site_ids=local)
    pos = np.searchsorted(local, sites)
    dual_b, site_b = sampler.boundary_draws(ref["p_dual"], ref["u_dual"], ref["cdf"], ref["u_site"], BOUNDARY_EPS)
    # a dual draw at its boundary may flip a bit: its endpoints are exempt
    exempt = site_b.copy()
    for c_, e_ in zip(*np.nonzero((dual_b & dec.active[None]).any(axis=2))):
        exempt[c_, dec.src[e_]] = True
        exempt[c_, dec.dst[e_]] = True
    got, want, ex = x1[:, sites], ref["x"][:, pos], exempt[:, pos]
    bad = (got != want) & ~ex
    print(mode, "sampled", got.size, "exempt", int(ex.sum()), "differing", int((got != want).sum()))
    assert not bad.any(), f"{int(bad.sum())} of {got.size} sampled labels differ away from boundaries"
    assert ex.sum() < 0.01 * ex.size
