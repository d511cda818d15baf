"""The seeded input generator: determinism, sizes and the structural invariants the tracker assumes."""
import numpy as np
import pytest

from paper_1711_07999_gb300 import synth


@pytest.mark.parametrize("cfg", [1, 2])
def test_model_is_deterministic_and_well_formed(cfg):
    a = synth.make_model(cfg)
    b = synth.make_model(cfg)
    for k in ("verts", "tris", "bone_idx", "bone_w"):
        assert np.array_equal(a["mesh"][k], b["mesh"][k])
    me, sk = a["mesh"], a["skeleton"]
    target = synth.CONFIGS[cfg]["V"]
    assert abs(len(me["verts"]) - target) <= 0.02 * target
    L = len(sk["parent"])
    assert L <= 72 and all(sk["parent"][j] < j for j in range(L))
    assert np.allclose(me["bone_w"].sum(1), 1.0, atol=1e-6)
    assert (me["bone_idx"] < L).all() and ((me["bone_w"] > 0).sum(1) <= 4).all()
    assert me["tris"].min() >= 0 and me["tris"].max() < len(me["verts"])
    # offsets are unit dual quaternions with identity rotation
    off = sk["offset_dq"]
    assert np.allclose(off[:, :4], [1, 0, 0, 0]) and np.allclose(off[:, 4], 0)


def test_seed_formula_and_sessions_differ():
    assert synth.seed_for(2, 5) == 17110799 + 2000 + 5
    a = synth.make_model(1, session=0)
    b = synth.make_model(1, session=1)
    assert not np.array_equal(a["mesh"]["verts"], b["mesh"]["verts"])


def test_noise_model():
    rng = np.random.default_rng(0)
    d = np.full((200, 300), 3.0, np.float32)
    d[:10] = 0
    n2 = synth.add_noise(d, 2, rng)
    valid = n2 > 0
    assert 0.015 < 1 - valid[10:].mean() < 0.025  # 2 % dropped
    assert abs(np.std(n2[valid] - 3.0) - 0.0015) < 1e-4
    n1 = synth.add_noise(d, 1, rng)
    q = n1[n1 > 0] * 1000
    assert np.allclose(q, np.round(q), atol=1e-3)  # quantised to 1 mm
