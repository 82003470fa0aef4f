"""GPU parity of the mass operator (kernel 6, the Laghos kernel of Sec. 5):
y_e = B^T diag(op_e) B x_e over a batch of elements, specialized on
(dimension, dofs per dimension D, quadrature points per dimension Q) and
generic, against the FP64 oracle (which forms the Kronecker product B
explicitly).  FP64 within 1e-12 and FP32 within 1e-5 relative Frobenius error
per element; element counts end in ragged tails of a block."""
import numpy as np
import pytest

import oracle
import synth
from paper_1904_08555_b300 import cj

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5


def tol32(dim, D, Q):
    """FP32 bound: each of the 2 dim stages is a dot product of length at most
    max(D, Q), whose rounding error is at most that length times the unit
    roundoff 2^-24 relative to the sum of |terms|; a factor 4 allows for the
    cancellation between terms.  At least 1e-5, the library's FP32 tolerance."""
    return max(TOL32, 4 * 2 * dim * max(D, Q) * 2.0 ** -24)


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cj.init(sync=True, compile_threads=4)
    yield
    cj.shutdown()


def run_mass(h, B1, op, x, dt):
    tdt = torch.float64 if dt == cj.F64 else torch.float32
    Bt = torch.from_numpy(B1).to("cuda", tdt)
    opt = torch.from_numpy(op).to("cuda", tdt)
    xt = torch.from_numpy(x).to("cuda", tdt)
    y = torch.full_like(xt, float("nan"))
    cj.launch_mass(h, Bt, opt, xt, y, x.shape[0])
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


def max_rel_err(y, ref):
    return float(np.max(np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)))


SHAPES = [(2, 1, 1), (2, 2, 3), (2, 3, 4), (2, 4, 6), (2, 5, 8), (2, 6, 3), (2, 16, 16),
          (3, 2, 3), (3, 3, 4), (3, 4, 6), (3, 5, 8), (3, 6, 5), (3, 8, 8)]


@pytest.mark.parametrize("dim,D,Q", SHAPES)
@pytest.mark.parametrize("dt", [cj.F64, cj.F32])
@pytest.mark.parametrize("generic", [False, True])
def test_mass_against_oracle(dim, D, Q, dt, generic):
    h = cj.specialize(cj.K_MASS, dt, n=D, m=Q, d=dim, flags=cj.FLAG_GENERIC if generic else 0)
    assert h.variant == ("generic" if generic else "jit")
    epb = max(1, 256 // max(D, Q) ** 2)
    ne = 5 * epb + 3                             # several blocks and a ragged last one
    B1, op, x = synth.mass_inputs_np(synth.SEED_MASS, dim, D, Q, ne)
    if dt == cj.F32:                             # the reference starts from the rounded inputs
        B1, op, x = (a.astype(np.float32).astype(np.float64) for a in (B1, op, x))
    ref = oracle.mass(B1, op, x, dim, nthreads=4)
    y = run_mass(h, B1, op, x, dt)
    assert np.all(np.isfinite(y))
    assert max_rel_err(y, ref) <= (TOL64 if dt == cj.F64 else tol32(dim, D, Q))


@pytest.mark.parametrize("dim,D,Q,epb", [(2, 3, 4, 1), (2, 4, 6, 3), (2, 4, 6, 16), (3, 3, 4, 2), (3, 5, 8, 1),
                                         (3, 4, 6, 7)])
def test_mass_explicit_tiles(dim, D, Q, epb):
    h = cj.specialize(cj.K_MASS, cj.F64, n=D, m=Q, d=dim, tile=(epb, 0, 0, 0))
    ne = 4 * epb + 1
    B1, op, x = synth.mass_inputs_np(synth.SEED_MASS, dim, D, Q, ne)
    ref = oracle.mass(B1, op, x, dim)
    assert max_rel_err(run_mass(h, B1, op, x, cj.F64), ref) <= TOL64


def test_mass_empty_batch_is_a_no_op():
    h = cj.specialize(cj.K_MASS, cj.F64, n=3, m=4, d=2)
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    cj.launch_mass(h, z, z, z, z, 0)
    torch.cuda.synchronize()


def test_mass_invalid_requests_are_refused():
    for kw in (dict(n=3, m=4, d=4), dict(n=17, m=4, d=2), dict(n=3, m=0, d=3)):
        with pytest.raises(cj.CJError) as e:
            cj.specialize(cj.K_MASS, cj.F64, **kw)
        assert e.value.status == cj.CJ_ERR_INVALID_ARG
    with pytest.raises(cj.CJError):
        cj.specialize(cj.K_MASS, cj.BF16, n=3, m=4, d=2)


@pytest.mark.parametrize("dim,D,Q,dt", [(2, 4, 6, cj.F64), (3, 4, 6, cj.F64), (3, 3, 4, cj.F32)])
def test_mass_full_size_sampled(dim, D, Q, dt):
    """The bench's sizes and launch configuration (the default tile), checked
    on 300 seeded elements against the oracle."""
    ne = (1 << 28) // (2 * D ** dim + Q ** dim) // 8
    tdt = torch.float64 if dt == cj.F64 else torch.float32
    B1, op, x = synth.mass_inputs_torch(synth.SEED_MASS, dim, D, Q, ne, "cuda")
    op, x = op.to(tdt), x.to(tdt)
    y = torch.empty_like(x)
    h = cj.specialize(cj.K_MASS, dt, n=D, m=Q, d=dim)
    Bt = torch.from_numpy(B1).to("cuda", tdt)
    cj.launch_mass(h, Bt, op, x, y, ne)
    torch.cuda.synchronize()
    rng = np.random.default_rng(9)
    idx = np.unique(np.concatenate([[0, ne - 1], rng.integers(0, ne, 300)]))
    it = torch.from_numpy(idx).cuda()
    ref = oracle.mass(Bt.double().cpu().numpy(), op[it].double().cpu().numpy(), x[it].double().cpu().numpy(), dim)
    assert max_rel_err(y[it].double().cpu().numpy(), ref) <= (TOL64 if dt == cj.F64 else TOL32)


PIPE_SHAPES = [(2, 2, 3), (2, 3, 4), (2, 5, 8), (2, 16, 16), (3, 2, 3), (3, 4, 6), (3, 5, 8), (3, 8, 8)]


@pytest.mark.parametrize("dim,D,Q", PIPE_SHAPES)
@pytest.mark.parametrize("dt", [cj.F64, cj.F32])
def test_mass_persistent_staged(dim, D, Q, dt):
    """Tile {epb, 1}: a persistent grid whose blocks stage the next group's x and
    op with cp.async while computing the current one.  Enough elements that every
    block runs several groups (the grid is at most 148 SMs x 8 blocks), with a
    ragged last group."""
    epb = max(1, 256 // max(D, Q) ** 2)
    h = cj.specialize(cj.K_MASS, dt, n=D, m=Q, d=dim, tile=(epb, 1, 0, 0))
    assert h.variant == "jit"
    ne = 3 * 148 * 8 * epb + 5
    B1, op, x = synth.mass_inputs_np(synth.SEED_MASS, dim, D, Q, ne)
    if dt == cj.F32:
        B1, op, x = (a.astype(np.float32).astype(np.float64) for a in (B1, op, x))
    ref = oracle.mass(B1, op, x, dim, nthreads=8)
    y = run_mass(h, B1, op, x, dt)
    assert np.all(np.isfinite(y))
    assert max_rel_err(y, ref) <= (TOL64 if dt == cj.F64 else tol32(dim, D, Q))


@pytest.mark.parametrize("ne", [1, 2, 5, 37])
def test_mass_persistent_small_batches(ne):
    """Fewer elements than one group, and fewer groups than blocks."""
    h = cj.specialize(cj.K_MASS, cj.F64, n=4, m=6, d=3, tile=(7, 1, 0, 0))
    B1, op, x = synth.mass_inputs_np(synth.SEED_MASS, 3, 4, 6, ne)
    ref = oracle.mass(B1, op, x, 3)
    assert max_rel_err(run_mass(h, B1, op, x, cj.F64), ref) <= TOL64


def test_mass_persistent_tile_is_validated():
    with pytest.raises(cj.CJError):
        cj.specialize(cj.K_MASS, cj.F64, n=4, m=6, d=3, tile=(7, 2, 0, 0))


THREAD_SHAPES = [(1, 1), (2, 2), (2, 3), (3, 4), (4, 6), (4, 8), (5, 8), (6, 3), (8, 2)]


@pytest.mark.parametrize("D,Q", THREAD_SHAPES)
@pytest.mark.parametrize("dt", [cj.F64, cj.F32])
@pytest.mark.parametrize("epb", [64, 128])
def test_mass_thread_per_element(D, Q, dt, epb):
    """Tile {epb, 2}: 2-D elements, one thread each, every stage in registers;
    several blocks and a ragged last one."""
    h = cj.specialize(cj.K_MASS, dt, n=D, m=Q, d=2, tile=(epb, 2, 0, 0))
    assert h.variant == "jit"
    ne = 5 * epb + 3
    B1, op, x = synth.mass_inputs_np(synth.SEED_MASS, 2, D, Q, ne)
    if dt == cj.F32:
        B1, op, x = (a.astype(np.float32).astype(np.float64) for a in (B1, op, x))
    ref = oracle.mass(B1, op, x, 2, nthreads=4)
    y = run_mass(h, B1, op, x, dt)
    assert np.all(np.isfinite(y))
    assert max_rel_err(y, ref) <= (TOL64 if dt == cj.F64 else tol32(2, D, Q))


def test_mass_thread_per_element_is_validated():
    with pytest.raises(cj.CJError):   # 3-D
        cj.specialize(cj.K_MASS, cj.F64, n=3, m=4, d=3, tile=(128, 2, 0, 0))
    with pytest.raises(cj.CJError):   # D Q + D^2 = 96 values per thread
        cj.specialize(cj.K_MASS, cj.F64, n=6, m=10, d=2, tile=(128, 2, 0, 0))
