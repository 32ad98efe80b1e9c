import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def tiny():
    import gen
    return gen.tiny_scene(), gen.tiny_camera()


def single_gaussian_model(o=0.5, col=(0.9, 0.4, 0.2), s_a=0.05, sig_s=0.5, z0=10.0,
                          pos=(0.0, 0.0), k=10):
    """One anchor at (x, y, z0) whose only kept Gaussian j=0 has opacity o,
    colour col, isotropic scale s_a*sig_s and identity rotation; the other
    Gaussians get a negative opacity bias and are dropped.  Layer-2 weights
    are zero, so the derived attributes equal the activations of the biases."""
    import gen
    W1, b1, W2, b2 = gen.glorot_mlps(5, k)
    W2 = [np.zeros_like(w) for w in W2]
    b2 = [np.zeros_like(b) for b in b2]
    b2[0][:] = -1.0
    b2[0][0] = np.arctanh(o)
    logit = lambda p: np.log(p / (1.0 - p))
    b2[1][0:3] = [logit(c) for c in col]
    b2[2][0:3] = logit(sig_s)
    b2[2][3:7] = [1.0, 0.0, 0.0, 0.0]
    b2 = [b.astype(np.float32) for b in b2]
    m = gen.Model(pos=np.array([[pos[0], pos[1], z0]], np.float32),
                  feat=np.zeros((1, 32), np.float32),
                  offs=np.zeros((1, k, 3), np.float32),
                  scale=np.array([s_a], np.float32), level=np.zeros(1, np.uint8),
                  n_levels=1, lod_dmax=0.0, W1=W1, b1=b1, W2=W2, b2=b2, k=k, name="single")
    m.validate()
    return m


def axis_camera(w=128, h=96, f=100.0):
    """Camera at the origin looking along +z (R = I)."""
    import gen
    return gen.Camera(R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), fx=f, fy=f,
                      cx=w / 2.0, cy=h / 2.0, width=w, height=h, znear=0.2)
