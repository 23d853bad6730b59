"""Sub-model of whole blocks of a learned-proposal model: the sampled blocks'
sites, every edge incident to them and the sites at the far ends.  A sampled
block's learned update (its cut duals, features, proposal and MH test) only
involves its sites and their incident edges, so on this sub-model the oracle
reproduces the full model's update of those blocks, given the full model's
edge slots, site ids and block ids as the draw contract's indices."""
import numpy as np

from paper_1611_06684_gb300 import workloads as wl


def learned_sub_model(model, block_of_site, blocks):
    """Returns (sub model, local -> global site ids, edge ids, sub block_of_site,
    local -> global block ids, number of sampled blocks); the sampled blocks
    are local blocks 0 .. k-1 in the given order, every other site a
    singleton block after them."""
    blocks = np.asarray(blocks, np.int64)
    sampled = np.isin(block_of_site, blocks)
    sites = np.nonzero(sampled)[0]
    inc = sampled[model.src] | sampled[model.dst]
    eids = np.nonzero(inc)[0]
    local = np.unique(np.concatenate([sites, model.src[eids], model.dst[eids]]))
    sub = wl.Model(n_vars=len(local), n_labels=model.n_labels, unary=model.unary[local],
                   src=np.searchsorted(local, model.src[eids]).astype(np.int32),
                   dst=np.searchsorted(local, model.dst[eids]).astype(np.int32),
                   pair=model.pair[eids], name="learned_sub")
    k = len(blocks)
    pos = {int(b): i for i, b in enumerate(blocks)}
    sub_bos = np.zeros(len(local), np.int64)
    block_ids = list(blocks)
    nxt = k
    for i, v in enumerate(local):
        b = int(block_of_site[v])
        if b in pos:
            sub_bos[i] = pos[b]
        else:
            sub_bos[i] = nxt
            block_ids.append(-1)                     # not compared
            nxt += 1
    return sub, local, eids, sub_bos, np.array(block_ids, np.int64), k
