"""Shared helpers of the tests (inputs, oracle runs, comparisons, paper fixtures)."""
import json
import os

import numpy as np

import paper_2404_02950_gb300 as slh
from oracle.eom import EOMParams as OParams


def golden(name):
    """A fixture of values the paper prints (tests/golden/; each file names its source)."""
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        return json.load(f)


def oparams(p: slh.EOMParams) -> OParams:
    return OParams(lam=p.lam, a=p.a, friction=p.friction, eta_power=p.eta_power, order=p.order,
                   ko_order=p.ko_order, ko_eps=p.ko_eps)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def uniform_hierarchy(n, dx, prec="f64", nghost=3, bf=8, boxes=None, fused_tags=False):
    boxes = boxes or [((0, 0, 0), (n - 1, n - 1, n - 1))]
    h = slh.Hierarchy(n, dx, nghost=nghost, bf=bf, prec=prec, max_levels=1)
    h.init_level(0, boxes, fused_tags=fused_tags)
    return h, boxes


def upload(h, lev, fields, boxes):
    h.set_state(lev, slh.dense_from_boxes(fields, boxes))


def download_domain(h, lev, boxes, n):
    """Dense valid cells -> four [z, y, x] domain arrays (level covering the domain)."""
    per = slh.boxes_from_dense(h.get_state(lev), boxes)
    out = [np.zeros((n, n, n)) for _ in range(4)]
    for (lo, hi), a in zip(boxes, per):
        for c in range(4):
            out[c][lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] = a[c]
    return out


def tags_domain(tags_dense, boxes, n):
    t = np.asarray(tags_dense)
    out = np.zeros((n, n, n), dtype=np.uint8)
    off = 0
    for lo, hi in boxes:
        sz = [hi[d] - lo[d] + 1 for d in range(3)]
        vol = sz[0] * sz[1] * sz[2]
        out[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] = t[off:off + vol].reshape(sz[2], sz[1], sz[0])
        off += vol
    return out


def box_padded_views(h, lev, role=None):
    """Per-box padded (slots, pnz, pny, pitch) torch views of a level buffer."""
    info = h.levels[lev]
    nc = h.nslots
    offs, geom, _, _ = slh.slh_level_layout(h.nghost, info["boxes"], nc)
    buf = h.state_buffer(lev) if role is None else info["bufs"][role]
    views = []
    for b in range(len(info["boxes"])):
        pitch, pny, pnz, cs = (int(v) for v in geom[b])
        o = int(offs[b])
        v = buf[o:o + nc * cs].view(nc, cs)[:, :pitch * pny * pnz].view(nc, pnz, pny, pitch)
        views.append(v)
    return views
