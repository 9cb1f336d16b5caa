"""Hand-made tiny scene batches shared by the tests."""
import numpy as np

import synth


def tiny_batch(objects, poly=((-1, -1), (1, -1), (1, 1), (-1, 1)), obbs=(), n_cand=1, rel=None, relp=None,
               dirs=None, anchors=None, parts=None, obb_part=None, part_q=None):
    """objects: list of sphere lists [(x,y,z,r), ...] in object frames; rel,
    relp, dirs, anchors: per-object relation fields (defaults: all free);
    parts [n][12], obb_part [n_obb], part_q [n_cand][n]: articulated parts."""
    n = len(objects)
    part_rows = parts
    parts = dict(
        sph=np.array([s for o in objects for s in o], np.float32), nsph=np.array([len(o) for o in objects]),
        half=np.array([[0.1, 0.1, 0.1, 0.15]] * n, np.float32),
        rel=np.zeros(n, np.int32) if rel is None else np.array(rel, np.int32),
        relp=np.tile(np.array([0.05, 0.2, 0.0, 0.0], np.float32), (n, 1)) if relp is None
        else np.array(relp, np.float32).reshape(n, 4),
        dir=np.zeros(n, np.float32) if dirs is None else np.array(dirs, np.float32),
        anchors=[[] for _ in range(n)] if anchors is None else [list(a) for a in anchors],
        poly=np.array(poly, np.float32), z=0.0, obb=np.array(obbs, np.float32).reshape(-1, 12), ncand=n_cand,
        base=np.zeros(4, np.float32))
    if part_rows is not None:
        parts["parts"] = np.array(part_rows, np.float32).reshape(-1, 12)
        parts["obb_part"] = (-np.ones(len(parts["obb"]), np.int32) if obb_part is None
                             else np.array(obb_part, np.int32))
        parts["part_q"] = (np.zeros((n_cand, len(parts["parts"])), np.float32) if part_q is None
                           else np.array(part_q, np.float32).reshape(n_cand, -1))
    return synth._pack([parts])


def cabinet_with_meshes(seed=11, n_templates=16, cand_per_template=8):
    """Cabinet templates (parts, INSIDE objects, part boxes) with a sphere
    mesh and a box mesh on the counter: every world feature in one batch."""
    rng = np.random.default_rng(seed)
    parts = []
    for _ in range(n_templates):
        p = synth.cabinet_template(rng, int(rng.integers(3, 7)), int(rng.integers(2, 4)), 1, 12)
        c1 = [rng.uniform(-0.25, 0.25), rng.uniform(-0.7, 0.7), 0.9 + rng.uniform(0.05, 0.2)]
        c2 = [rng.uniform(-0.25, 0.25), rng.uniform(-0.7, 0.7), 0.95]
        p["tri"] = np.concatenate([synth.sphere_mesh(c1, rng.uniform(0.05, 0.12)),
                                   synth.box_mesh(c2, np.eye(3), rng.uniform(0.03, 0.1, 3))]).astype(np.float32)
        p["ncand"] = cand_per_template
        nd = len(p["parts"])
        p["part_q"] = (p["parts"][:, 3] + (p["parts"][:, 4] - p["parts"][:, 3]) *
                       rng.uniform(size=(cand_per_template, nd))).astype(np.float32)
        parts.append(p)
    return synth._pack(parts, name="cabinet+meshes")
