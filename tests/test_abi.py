"""The C-ABI library loads, exports every symbol include/sceniris.h declares,
and its host-only paths (argument validation, the LPT ordering helper) work
without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from paper_2512_16896_b300 import _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(sc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    from paper_2512_16896_b300 import build
    build.build()
    return _native.lib()


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n
    # and the binding mirrors each of them
    assert set(names) <= set(_native.SIGNATURES), set(names) - set(_native.SIGNATURES)


def test_version_and_error_string(L):
    assert L.sc_version() >= 100
    assert isinstance(L.sc_last_error(), bytes)


def test_invalid_arguments_rejected_before_launch(L):
    """NULL context / outputs are refused on the host with SC_ERR_INVALID and a message."""
    assert L.sc_sample_poses(None, None, None, None, 0, None, None, None) == _native.SC_ERR_INVALID
    assert b"ctx" in L.sc_last_error()
    assert L.sc_collide(None, None, None, None, 0, 0, None, None, None) == _native.SC_ERR_INVALID
    assert L.sc_ctx_create(0, None, None) == _native.SC_ERR_INVALID
    assert L.sc_ctx_set_stream(None, None) == _native.SC_ERR_INVALID
    assert L.sc_order_by_work(0, None, None, None, None) == _native.SC_ERR_INVALID


def test_order_by_work_is_lpt():
    b = synth.ragged(seed=5, n_templates=40, cand_per_template=3)
    order = _native.order_by_work(b)
    assert sorted(order.tolist()) == list(range(b.n_cand))
    t_of = b.cand_template()
    S = b.sphere_count_of_template().astype(np.float64)
    sq = np.array([np.sum(np.diff(b.obj_sph_off[b.tmpl_obj_off[t]:b.tmpl_obj_off[t + 1] + 1]).astype(np.float64) ** 2)
                   for t in range(b.n_templates)])
    work = 0.5 * (S * S - sq)
    w = work[t_of[order]]
    assert np.all(np.diff(w) <= 0)


def test_device_batch_checks_joint_value_shape():
    """The binding refuses joint values that do not cover every candidate's
    part slots (the library would read past them); no GPU needed: the check
    runs before any copy."""
    import numpy as np
    import pytest
    import synth
    from paper_2512_16896_b300 import _native
    b = synth.cabinet(seed=1, n_templates=2, cand_per_template=3)
    b.part_q = np.zeros((b.n_cand - 1, b.part_q.shape[1]), np.float32)
    with pytest.raises(ValueError):
        _native.DeviceBatch(b, device="cpu")


def test_device_batch_checks_mesh_and_part_offsets():
    """Triangle and part offsets must end at their array's length, obb_part
    must cover every box (checked in the binding before any copy)."""
    import numpy as np
    import pytest
    import synth
    from paper_2512_16896_b300 import _native
    m = synth.meshes(seed=1, n_templates=2, cand_per_template=2)
    m.tmpl_tri_off = m.tmpl_tri_off.copy()
    m.tmpl_tri_off[-1] += 1
    with pytest.raises(ValueError):
        _native.DeviceBatch(m, device="cpu")
    c = synth.cabinet(seed=1, n_templates=2, cand_per_template=2)
    c.obb_part = c.obb_part[:-1]
    with pytest.raises(ValueError):
        _native.DeviceBatch(c, device="cpu")
