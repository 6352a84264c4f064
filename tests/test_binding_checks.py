"""The Python binding refuses arrays whose sizes differ from what the library
will read or write, before any call crosses the C ABI (the ABI takes plain
pointers and cannot check them; a short device array would be overrun by a
kernel).  No GPU: a handle with a NULL context stands in, so arrays of the
right size reach the library and come back as FS_EINVAL (host arrays) or
fail the CUDA-tensor check (CPU tensors)."""
import ctypes

import numpy as np
import pytest

import paper_1602_05650_gb300 as fs
from paper_1602_05650_gb300 import build

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


@pytest.fixture
def h():
    # 3 fibers x 8 points, a 12-node surface (36 unknowns), no real context
    return fs.Handle(ctypes.c_void_p(0), 24, 4 * 24 + 36, 3)


def t(*shape, dtype=torch.float64):
    return torch.zeros(shape, dtype=dtype)


def test_state_arrays(h):
    with pytest.raises(ValueError, match="X has"):
        fs.fs_set_state(h, np.zeros((23, 3)), np.ones(3))
    with pytest.raises(ValueError, match="lengths"):
        fs.fs_set_state(h, np.zeros((24, 3)), np.ones(2))
    with pytest.raises(ValueError, match="f_ext"):
        fs.fs_set_state(h, np.zeros((24, 3)), np.ones(3), np.zeros((24, 2)))
    with pytest.raises(fs.FsError):                      # right sizes: the NULL context is refused
        fs.fs_set_state(h, np.zeros((24, 3)), np.ones(3), np.zeros((24, 3)))
    with pytest.raises(ValueError, match="T has"):
        fs.fs_get_state(h, T=np.zeros(23))
    with pytest.raises(ValueError, match="V has"):
        fs.fs_get_state(h, V=np.zeros((24, 2)))
    with pytest.raises(fs.FsError):
        fs.fs_get_state(h, X=np.zeros((24, 3)), T=np.zeros(24), V=np.zeros((24, 3)))


def test_growth_and_lengths(h):
    with pytest.raises(ValueError, match="Ldot"):
        fs.fs_set_growth(h, np.zeros(4))
    with pytest.raises(fs.FsError):
        fs.fs_set_growth(h, np.zeros(3))
    with pytest.raises(ValueError, match="3 fibers"):
        fs.fs_get_lengths(h, 5)
    with pytest.raises(fs.FsError):
        fs.fs_get_lengths(h, 3)


@pytest.mark.parametrize("apply", [fs.fs_stokeslet_apply, fs.fs_stokeslet_apply_tree])
def test_pair_sums(h, apply):
    X, T = t(10, 3), t(7, 3)
    bad = [((t(30), t(10, 3), T, t(7, 3)), "src_xyz"),           # flattened points
           ((X, t(9, 3), T, t(7, 3)), "src_wf"),
           ((X, t(10, 3), T, t(6, 3)), "out"),
           ((X, t(10, 3), t(7, 2), t(7, 3)), "tgt_xyz")]
    for args, name in bad:
        with pytest.raises(ValueError, match=name):
            apply(h, *args)
    with pytest.raises(ValueError, match="src_fiber"):
        apply(h, X, t(10, 3), T, t(7, 3), t(9, dtype=torch.int32), t(7, dtype=torch.int32))
    with pytest.raises(TypeError, match="CUDA tensor"):        # right sizes, CPU tensors
        apply(h, X, t(10, 3), T, t(7, 3), t(10, dtype=torch.int32), t(7, dtype=torch.int32))


def test_stresslet_and_surface(h):
    X, T = t(12, 3), t(5, 3)
    with pytest.raises(ValueError, match="src_w"):
        fs.fs_stresslet_apply(h, X, t(12, 3), t(11), t(12, 3), T, t(5, 3))
    with pytest.raises(ValueError, match="src_q"):
        fs.fs_stresslet_apply(h, X, t(12, 3), t(12), t(12, 2), T, t(5, 3))
    with pytest.raises(TypeError, match="CUDA tensor"):
        fs.fs_stresslet_apply(h, X, t(12, 3), t(12), t(12, 3), T, t(5, 3))
    with pytest.raises(ValueError, match="q has"):
        fs.fs_surface_apply(h, t(35), t(36))
    with pytest.raises(ValueError, match="out has"):
        fs.fs_surface_apply(h, t(12, 3), t(12, 2))
    with pytest.raises(TypeError, match="CUDA tensor"):
        fs.fs_surface_apply(h, t(12, 3), t(36))


def test_dynamic_instability_inputs():
    with pytest.raises(ValueError, match="lengths"):
        fs.fs_dynamic_instability([1, 1], [1.0], [0.5, 0.5], 0.1, 1.0, 1.0, 1.0, 1.0, 0.1)
    with pytest.raises(ValueError, match="u has"):
        fs.fs_dynamic_instability([1, 1], [1.0, 1.0], [0.5], 0.1, 1.0, 1.0, 1.0, 1.0, 0.1)


def test_constructors_and_submit():
    import workloads as wl
    b = wl.sphere_quadrature(6.0, 2, 4)
    short = wl.Boundary(b.R, b.nodes, b.normals, b.weights[:-1])
    with pytest.raises(ValueError, match="boundary weights"):
        fs.fs_create([8, 8], 1.0, 1e-3, 1.0, 1e-3, boundary=short)
    if not torch.cuda.is_available():
        with pytest.raises(fs.FsError):                  # right sizes: no CUDA device here
            fs.fs_create([8, 8], 1.0, 1e-3, 1.0, 1e-3, boundary=b)
    body = wl.sphere_body((0.0, 0.0, 0.0), 1.0, 2, 4)
    with pytest.raises(ValueError, match="minus_end"):
        fs.fs_create_with_body([8, 8], [1], 1.0, 1e-3, 1.0, 1e-3, body)
    bad_body = wl.RigidBody(body.centre, body.radius, body.nodes, body.normals[:-1], body.weights,
                            body.force, body.torque)
    with pytest.raises(ValueError, match="body normals"):
        fs.fs_create_with_body([8, 8], [1, 1], 1.0, 1e-3, 1.0, 1e-3, bad_body)
    bad_load = wl.RigidBody(body.centre, body.radius, body.nodes, body.normals, body.weights,
                            np.zeros(2), body.torque)
    with pytest.raises(ValueError, match="body force"):
        fs.fs_create_with_body([8, 8], [1, 1], 1.0, 1e-3, 1.0, 1e-3, bad_load)
    sv = fs.Server(ctypes.c_void_p(0))
    with pytest.raises(ValueError, match="X has"):
        fs.fs_submit(sv, [8, 8], np.zeros((15, 3)), [1.0, 1.0], 1.0, 1e-3, 1.0, 1e-3)
    with pytest.raises(ValueError, match="lengths"):
        fs.fs_submit(sv, [8, 8], np.zeros((16, 3)), [1.0], 1.0, 1e-3, 1.0, 1e-3)
    with pytest.raises(fs.FsError):                      # right sizes: the NULL server is refused
        fs.fs_submit(sv, [8, 8], np.zeros((16, 3)), [1.0, 1.0], 1.0, 1e-3, 1.0, 1e-3)
    with pytest.raises(ValueError, match="points_per_fiber"):
        fs.fs_create_batch([2, 3], [8] * 4, 1.0, 1e-3, 1.0, 1e-3)
