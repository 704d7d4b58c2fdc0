"""The boundary's handle calls on the GPU: vectors (create, wrap, set, get),
the solve on vector handles against the raw-pointer form, matrices with FP64
storage only, and checkpoints of the learned stage's network that resume
training exactly."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsv():
    from tests.helpers import build_library
    build_library()
    import paper_1602_05901_gb300 as m
    return m


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_vector_create_set_get_round_trip(rsv, torch, precision):
    nx, ny, nz = 7, 5, 3
    v = rsv.Vector.create(nx, ny, nz, precision=precision)
    assert v.n == 3 * nx * ny * nz
    assert np.array_equal(v.get(), np.zeros(v.n))  # created zeroed
    x = np.random.default_rng(1).standard_normal(v.n)
    ref = x if precision == "fp64" else x.astype(np.float32).astype(np.float64)
    v.set(x)
    assert np.array_equal(v.get(), ref)
    # device source and destination
    xd = torch.from_numpy(x).cuda()
    v.set(torch.zeros_like(xd))
    v.set(xd)
    out = torch.empty_like(xd)
    v.get(out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)


def test_vector_wrap_borrows_tensor_memory(rsv, torch):
    t = torch.arange(30, dtype=torch.float64, device="cuda")
    v = rsv.Vector.wrap(t)
    assert v.data_ptr == t.data_ptr() and v.n == 30 and v.precision == rsv.RSV_PREC_FP64
    v.set(np.full(30, 2.5))
    assert float(t.sum()) == 75.0
    t32 = torch.zeros(12, dtype=torch.float32, device="cuda")
    assert rsv.Vector.wrap(t32).precision == rsv.RSV_PREC_MIXED
    h = ctypes.c_void_p()
    host = np.zeros(8)
    # a host pointer is not device memory
    assert rsv.rsv_vec_wrap(ctypes.c_void_p(host.ctypes.data), 8, rsv.RSV_PREC_FP64, ctypes.byref(h)) == rsv.RSV_EINVAL
    # misaligned for float64
    assert rsv.rsv_vec_wrap(ctypes.c_void_p(t.data_ptr() + 4), 4, rsv.RSV_PREC_FP64, ctypes.byref(h)) == rsv.RSV_EINVAL


def test_solve_on_vector_handles_equals_raw_pointer_form(rsv, torch):
    p = synth.make_problem(20, 20, 10, seed=0)
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(p.vals)
    s = rsv.Solver(A, solver="gmres")
    s.setup("bilu0")
    # owned vectors, filled from the host
    b = rsv.Vector.create(p.nx, p.ny, p.nz)
    x = rsv.Vector.create(p.nx, p.ny, p.nz)
    b.set(p.b)
    info = rsv.rsv_solve_info()
    assert rsv.rsv_solve(s.handle, b.handle, x.handle, ctypes.byref(info)) == rsv.RSV_OK
    xv = x.get()
    # raw pointers, host buffers
    xh = np.zeros(p.n)
    info2 = rsv.rsv_solve_info()
    assert rsv.rsv_solve_ptr(s.handle, p.b.ctypes.data, xh.ctypes.data, 0, ctypes.byref(info2)) == rsv.RSV_OK
    assert info.iters == info2.iters and np.array_equal(xv, xh)
    relres = np.linalg.norm(p.b - oracle.spmv(p.row_ptr, p.col_idx, p.vals, xv)) / np.linalg.norm(p.b)
    assert relres <= 1e-8
    # wrong length, wrong precision, b and x the same vector
    short = rsv.Vector.create(p.nx, p.ny, p.nz - 1)
    x32 = rsv.Vector.create(p.nx, p.ny, p.nz, precision="mixed")
    assert rsv.rsv_solve(s.handle, short.handle, x.handle, None) == rsv.RSV_EINVAL
    assert rsv.rsv_solve(s.handle, b.handle, x32.handle, None) == rsv.RSV_EINVAL
    assert rsv.rsv_solve(s.handle, b.handle, b.handle, None) == rsv.RSV_EINVAL


def test_fp64_only_matrix(rsv, torch):
    p = synth.make_problem(9, 7, 5, seed=3)
    A = rsv.Matrix(p.nx, p.ny, p.nz, precision="fp64")
    A.set_values(p.vals)
    with pytest.raises(rsv.RsvError) as e:
        rsv.Solver(A, precision="mixed")
    assert e.value.status == rsv.RSV_EINVAL
    x32 = torch.zeros(p.n, dtype=torch.float32, device="cuda")
    assert rsv.rsv_spmv_f32(A.handle, 1.0, x32.data_ptr(), 0.0, x32.data_ptr()) == rsv.RSV_EINVAL
    s = rsv.Solver(A, solver="gmres")
    s.setup("cpr")
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros_like(b)
    st, info = s.solve(b, x)
    assert st == rsv.RSV_OK and info["true_relres"] <= 1e-8


def test_unet_checkpoint_resumes_training_bit_exactly(rsv, torch, tmp_path):
    """Train a network, save it (weights, Adam moments, step), train on; a fresh
    network loaded from the checkpoint and trained on the same samples ends with
    bit-identical weights."""
    nx, ny, nz, base, levels = 32, 8, 8, 32, 2
    rng = np.random.default_rng(5)
    V = nx * ny * nz
    samples = [tuple(torch.tensor(rng.standard_normal(V) * sc, device="cuda") for sc in (3.0, 1.0, 0.5))
               for _ in range(6)]
    rps, lnks, tgts = zip(*samples)
    net = rsv.Unet(nx, ny, nz, base=base, levels=levels)
    net.set_params(synth.unet_init(base, levels, seed=1))
    net.train_batch(rps[:3], lnks[:3], tgts[:3], 1e-3)
    ck = tmp_path / "net.rsvunet"
    net.save(str(ck))
    head = open(ck, "rb").read(200)
    assert head.startswith(b"RSVUNET1\n{\"format\":\"rsv_unet\"") and b"\"adam_step\":3" in head
    l1 = net.train_batch(rps[3:], lnks[3:], tgts[3:], 1e-3)
    p1 = net.params()
    net2 = rsv.Unet(nx, ny, nz, base=base, levels=levels)
    net2.load(str(ck))
    l2 = net2.train_batch(rps[3:], lnks[3:], tgts[3:], 1e-3)
    p2 = net2.params()
    assert np.array_equal(l1, l2) and np.array_equal(p1, p2)
    # without the three steps before the checkpoint the weights differ
    net3 = rsv.Unet(nx, ny, nz, base=base, levels=levels)
    net3.set_params(synth.unet_init(base, levels, seed=1))
    net3.train_batch(rps[3:], lnks[3:], tgts[3:], 1e-3)
    assert not np.array_equal(net3.params(), p1)
    # another architecture, a truncated file: EINVAL, network unchanged
    other = rsv.Unet(nx, ny, nz, base=base, levels=1)
    with pytest.raises(rsv.RsvError) as e:
        other.load(str(ck))
    assert e.value.status == rsv.RSV_EINVAL
    data = open(ck, "rb").read()
    bad = tmp_path / "cut.rsvunet"
    open(bad, "wb").write(data[:-4])
    with pytest.raises(rsv.RsvError):
        net2.load(str(bad))
    assert np.array_equal(net2.params(), p2)
