"""trk_create refuses malformed models before it touches the device (host logic: runs with or without a
GPU).  Each case damages one field of a valid model and checks the status and the message naming it;
failure detection is exercised on the host, with no device fault."""
import copy
import os
import re

import numpy as np
import pytest

from paper_1711_07999_gb300 import synth, trk


def _model():
    return synth.make_model(1, V=500, width=48)


def _set(path, value):
    def f(m):
        d = m
        for k in path[:-1]:
            d = d[k]
        d[path[-1]] = value
    return f


def _edit(part, key, fn):
    def f(m):
        a = np.array(m[part][key], copy=True)
        fn(a)
        m[part][key] = a
    return f


def _long_chain(m):
    n = trk_max_links() + 1
    m["skeleton"] = dict(parent=np.arange(-1, n - 1), type=np.zeros(n, np.int32),
                         axis=np.tile([0.0, 0.0, 1.0], (n, 1)), offset_dq=np.tile([1.0, 0, 0, 0, 0, 0, 0, 0], (n, 1)),
                         prior_mask=np.ones(n))


def trk_max_links():
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "trk.h")
    return int(re.search(r"#define TRK_MAX_LINKS (\d+)", open(hdr).read()).group(1))


def _unit_dual_not_orthogonal(a):
    a[1, 4:] += 0.1 * a[1, :4]  # <real, dual> = 0.1 |real|^2: not a rigid motion


CASES = [
    ("triangle index past the vertices", _edit("mesh", "tris", lambda a: a.__setitem__((5, 1), 496)),
     trk.TRK_ERR_INVALID_ARG, "tris[16] out of range"),
    ("negative triangle index", _edit("mesh", "tris", lambda a: a.__setitem__((0, 0), -1)),
     trk.TRK_ERR_INVALID_ARG, "tris[0] out of range"),
    ("weights not summing to one", _edit("mesh", "bone_w", lambda a: a.__setitem__(7, a[7] * 0.9)),
     trk.TRK_ERR_INVALID_ARG, "weights of vertex 7"),
    ("negative weight", _edit("mesh", "bone_w", lambda a: a.__setitem__((3, 1), -0.25)),
     trk.TRK_ERR_INVALID_ARG, "bone slot 1 of vertex 3"),
    ("bone index past the links", _edit("mesh", "bone_idx", lambda a: a.__setitem__((9, 0), 31)),
     trk.TRK_ERR_INVALID_ARG, "bone slot 0 of vertex 9"),
    ("non-finite vertex", _edit("mesh", "verts", lambda a: a.__setitem__((11, 2), np.nan)),
     trk.TRK_ERR_NUMERIC, "vertex 11 not finite"),
    ("parent after its child", _edit("skeleton", "parent", lambda a: a.__setitem__(3, 3)),
     trk.TRK_ERR_INVALID_ARG, "parent[3]"),
    ("parent below -1", _edit("skeleton", "parent", lambda a: a.__setitem__(0, -2)),
     trk.TRK_ERR_INVALID_ARG, "parent[0]"),
    ("unknown joint type", _edit("skeleton", "type", lambda a: a.__setitem__(2, 2)),
     trk.TRK_ERR_INVALID_ARG, "type[2]"),
    ("zero joint axis", _edit("skeleton", "axis", lambda a: a.__setitem__(1, 0.0)),
     trk.TRK_ERR_INVALID_ARG, "axis[1] not unit"),
    ("offset of non-unit norm", _edit("skeleton", "offset_dq", lambda a: a.__setitem__((1, slice(0, 4)), a[1, :4] * 1.1)),
     trk.TRK_ERR_INVALID_ARG, "offset_dq[1] not unit"),
    ("offset that is no rigid motion", _edit("skeleton", "offset_dq", _unit_dual_not_orthogonal),
     trk.TRK_ERR_INVALID_ARG, "offset_dq[1] not unit"),
    ("non-finite prior mask", _edit("skeleton", "prior_mask", lambda a: a.__setitem__(4, np.nan)),
     trk.TRK_ERR_INVALID_ARG, "prior_mask[4]"),
    ("zero focal length", _set(("camera", "fx"), 0.0), trk.TRK_ERR_INVALID_ARG, "bad intrinsics"),
    ("non-finite principal point", _set(("camera", "cy"), float("nan")), trk.TRK_ERR_INVALID_ARG, "bad intrinsics"),
    ("image above 2^28 pixels", lambda m: m["camera"].update(width=20000, height=20000),
     trk.TRK_ERR_NO_CAPACITY, "image too large"),
    ("more links than the limit", _long_chain, trk.TRK_ERR_NO_CAPACITY, f"n_links {trk_max_links() + 1} >"),
]


@pytest.mark.parametrize("name, damage, status, msg", CASES, ids=[c[0] for c in CASES])
def test_malformed_model_is_refused(name, damage, status, msg):
    m = copy.deepcopy(_model())
    damage(m)
    with pytest.raises(trk.TrkError) as e:
        trk.Session(m)
    assert e.value.status == status
    assert msg in str(e.value)
