"""The C boundary's field-order conversions and its latched device status.

* fl_mesh_to_internal / fl_mesh_to_user move cell and face fields of a
  renumbered mesh between the caller's numbering and the library's, in one
  gather or scatter kernel: checked element for element against the
  published permutation (fl_mesh_permutation), as a round trip, and as a
  plain copy for meshes that were not renumbered.
* A device-side error recorded by a kernel (a bounded wait that gave up)
  is returned by the next call on the mesh, which then runs nothing, and
  once only; fl_mesh_status returns it after synchronising.  The error is
  recorded by a small probe kernel (tests/cuda/status_probe.cu) through the
  same device store the library's kernels use: no wait is made to expire."""
import ctypes
import os
import subprocess

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2110_03044_gb300", "csrc")


def _meshes():
    return {"hex_permuted": W.permuted_mesh(W.structured_mesh(11, 7, 5, 0.1, 0.2, 0.3), 3)[0],
            "tet": W.tet_mesh(4)}


@pytest.mark.parametrize("name", ["hex_permuted", "tet"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("renumber", [True, False])
def test_reorder_matches_published_permutation(fl, name, dtype, renumber):
    mesh = _meshes()[name]
    m = fl.Mesh.from_faces(mesh.n_cells, mesh.face_cells, mesh.normals, mesh.areas,
                           mesh.volumes, renumber=renumber)
    cp, fp, flip = m.permutation()
    assert not flip.any()
    if not renumber:
        assert np.array_equal(cp, np.arange(mesh.n_cells))
    rng = np.random.default_rng(5)
    for kind, n, perm in (("cell", mesh.n_cells, cp), ("face", mesh.n_faces, fp)):
        x = rng.standard_normal(n)
        xd = torch.tensor(x, dtype=dtype, device="cuda")
        xi = m.to_internal(xd, kind)
        want = np.empty(n)
        want[perm] = x.astype(np.float32 if dtype == torch.float32 else np.float64)
        assert np.array_equal(xi.cpu().double().numpy(), want)
        back = m.to_user(xi, kind)
        assert torch.equal(back, xd)
    m.close()


def test_reorder_on_structured_mesh_is_a_copy_and_rejects_aliasing(fl):
    m = fl.Mesh.structured(9, 4, 3, 1.0, 1.0, 1.0)
    x = torch.arange(m.n_cells, dtype=torch.float64, device="cuda")
    assert torch.equal(m.to_internal(x, "cell"), x)
    u = torch.arange(m.n_faces, dtype=torch.float32, device="cuda")
    assert torch.equal(m.to_user(u, "face"), u)
    with pytest.raises(fl.FLError) as e:
        fl.fl_mesh_to_internal(m.handle, "cell", torch.float64, x, x)
    assert e.value.status == fl.FL_EINVAL
    # an unknown field kind is refused by the library itself
    st = fl.lib().fl_mesh_to_user(m.handle, 7, fl.FL_F64, x.data_ptr(),
                                  torch.empty_like(x).data_ptr(), None)
    assert st == fl.FL_EINVAL
    m.close()


@pytest.fixture(scope="module")
def status_probe(tmp_path_factory):
    from paper_2110_03044_gb300._build_lib import ARCH, INCLUDE, _nvcc
    out = str(tmp_path_factory.mktemp("probe") / "status_probe.so")
    cmd = [_nvcc()] + ARCH + ["-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                              "-I" + CSRC, "-I" + INCLUDE,
                              os.path.join(HERE, "cuda", "status_probe.cu"), "-o", out]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-3000:]
    lib = ctypes.CDLL(out)
    lib.probe_record_status.argtypes = [ctypes.c_void_p, ctypes.c_int]
    return lib


@pytest.mark.parametrize("kind", ["structured", "face_based"])
def test_recorded_device_error_is_returned_by_the_next_call(fl, status_probe, kind):
    if kind == "structured":
        m = fl.Mesh.structured(16, 8, 4, 0.1, 0.1, 0.1)
    else:
        mesh = W.structured_mesh(6, 5, 4, 0.1, 0.1, 0.1)
        m = fl.Mesh.from_faces(mesh.n_cells, mesh.face_cells, mesh.normals, mesh.areas,
                               mesh.volumes, renumber=True)
    th0 = torch.linspace(0, 1, m.n_cells, dtype=torch.float64, device="cuda")
    th = th0.clone()
    u = torch.full((m.n_faces,), 0.3, dtype=torch.float64, device="cuda")
    ws, nb = fl.workspace_for(m, torch.float64, 3)
    assert status_probe.probe_record_status(m.handle, fl.FL_ETIMEOUT) == 0
    with pytest.raises(fl.FLError) as e:
        fl.fl_step_rk(m.handle, "superbee", torch.float64, 3, 0.01, 2, th, u, ws, nb)
    assert e.value.status == fl.FL_ETIMEOUT
    assert "earlier call" in str(e.value)
    torch.cuda.synchronize()
    assert torch.equal(th, th0)  # the refused call ran nothing
    # returned once: the next call runs
    fl.fl_step_rk(m.handle, "superbee", torch.float64, 3, 0.01, 2, th, u, ws, nb)
    fl.fl_mesh_status(m.handle)
    # the synchronising query reports a recorded error the same way
    assert status_probe.probe_record_status(m.handle, fl.FL_ETIMEOUT) == 0
    with pytest.raises(fl.FLError) as e:
        fl.fl_mesh_status(m.handle)
    assert e.value.status == fl.FL_ETIMEOUT
    fl.fl_mesh_status(m.handle)
    m.close()
