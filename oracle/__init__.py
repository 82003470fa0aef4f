"""CPU oracle for the runtime-specialized kernels -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg
may import this package.  The product path (``paper_1904_08555_b300``) never
imports it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain scalar FP64 C, -ffp-contract=off);
this module only builds it with gcc and marshals numpy arrays.  Key encoding
(``keys.py``) is pure Python and holds only the key contract (byte format,
zeroed fields, flags, the variant rule), no rule for choosing a tile.

Pinning status (all pinned by CPU tests under tests/test_oracle_*.py):
  update_chain   -- zero input, identity, diagonal, binary-powering closed
                    form, exact rational brute force, commutation, layout.
  ltimes         -- six-order agreement, L=[I|0], L=0, in=1, numpy GEMM,
                    exact rational brute force.
  lplustimes     -- adjoint identity with ltimes, accumulation, numpy GEMM.
  mlp            -- central finite differences, linear least-squares closed
                    form, first Adam step closed form.
  eigen_bench    -- exact rational brute force for tiny sizes.
  eigen_recurrence -- the same recurrence over a batch of starts and any c.
  keys           -- keys assembled by hand from the documented byte format;
                    the variant rule against its statement.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11", "-pthread"]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, no vectorisation pragmas)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", *CFLAGS, "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def _bind(lib):
    """Argument and result types of the oracle's C functions on a loaded library
    (the tests also bind copies of oracle.c built with a planted mistake)."""
    P = ctypes.c_void_p
    i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.oracle_update_chain.argtypes = [i32, i32, i32, i64, P, P, i32]
    lib.oracle_update_chain.restype = i32
    lib.oracle_update_chain_uneven.argtypes = [i64, P, P, P, P, P]
    lib.oracle_update_chain_uneven.restype = i32
    lib.oracle_ltimes.argtypes = [i32, i32, i64, i64, i32, i32, P, P, P, i32]
    lib.oracle_ltimes.restype = i32
    lib.oracle_ltimes_sample.argtypes = [i32, i32, i64, i64, i32, P, P, i64, P, P]
    lib.oracle_lplustimes.argtypes = [i32, i32, i64, i64, i32, i32, P, P, P]
    lib.oracle_lplustimes.restype = i32
    lib.oracle_ltimes_sample.restype = i32
    lib.oracle_mlp_forward.argtypes = [i32, i32, i64] + [P] * 10
    lib.oracle_mlp_forward.restype = None
    lib.oracle_mlp_loss_grad.argtypes = [i32, i32, i64] + [P] * 14
    lib.oracle_mlp_loss_grad.restype = f64
    lib.oracle_adam.argtypes = [i64, P, P, P, P, i64, f64, f64, f64, f64]
    lib.oracle_adam.restype = None
    lib.oracle_eigen_bench.argtypes = [i32, i32, P]
    lib.oracle_eigen_bench.restype = None
    lib.oracle_eigen_recurrence.argtypes = [ctypes.c_longlong, i32, i32, ctypes.c_double, P, P]
    lib.oracle_eigen_recurrence.restype = None
    lib.oracle_mass.argtypes = [i32, i32, i32, i64, P, P, P, P, i32]
    lib.oracle_mass.restype = i32
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def update_chain(A: np.ndarray, steps: int, layout: int = 0, nthreads: int = 1) -> np.ndarray:
    """X_T for every instance of A (shape (batch, N, N), physical layout)."""
    A = _f64(A)
    batch, n, n2 = A.shape
    assert n == n2
    X = np.empty_like(A)
    rc = _load().oracle_update_chain(n, steps, layout, batch, _p(A), _p(X), nthreads)
    if rc != 0:
        raise ValueError("oracle_update_chain: invalid arguments")
    return X


def update_chain_uneven(n: np.ndarray, t: np.ndarray, offsets: np.ndarray,
                        A_pool: np.ndarray, nthreads: int = 1) -> np.ndarray:
    """X pool of the uneven chain.  nthreads > 1 splits the instance list into
    contiguous slices run by host threads (the foreign call releases the
    interpreter lock); instances are independent and each slice writes only
    its own instances, so the arithmetic is unchanged."""
    n = np.ascontiguousarray(n, dtype=np.int64)
    t = np.ascontiguousarray(t, dtype=np.int64)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    A_pool = _f64(A_pool)
    X_pool = np.zeros_like(A_pool)
    lib = _load()

    def run(k0, k1):
        return lib.oracle_update_chain_uneven(k1 - k0, _p(n[k0:]), _p(t[k0:]), _p(offsets[k0:]), _p(A_pool),
                                              _p(X_pool))

    nthreads = max(1, min(int(nthreads), len(n)))
    if nthreads == 1:
        rcs = [run(0, len(n))]
    else:
        from concurrent.futures import ThreadPoolExecutor
        bounds = [len(n) * i // nthreads for i in range(nthreads + 1)]
        with ThreadPoolExecutor(nthreads) as ex:
            rcs = list(ex.map(run, bounds[:-1], bounds[1:]))
    if any(rc != 0 for rc in rcs):
        raise ValueError("oracle_update_chain_uneven: invalid arguments")
    return X_pool


def ltimes(L: np.ndarray, x_phys: np.ndarray, G: int, Z: int, layout_in: int,
           layout_out: int, nthreads: int = 1) -> np.ndarray:
    """Physical out buffer (M*G*Z doubles, layout_out) from physical in."""
    L = _f64(L)
    x_phys = _f64(x_phys)
    M, D = L.shape
    out = np.empty(M * G * Z, dtype=np.float64)
    rc = _load().oracle_ltimes(M, D, G, Z, layout_in, layout_out, _p(L), _p(x_phys), _p(out), nthreads)
    if rc != 0:
        raise ValueError("oracle_ltimes: invalid arguments")
    return out


def lplustimes(Lp: np.ndarray, out_phys: np.ndarray, in_phys: np.ndarray, G: int, Z: int,
               layout_in: int, layout_out: int) -> np.ndarray:
    """in + Lp-contraction of out (new physical `in` buffer; Lp is [D][M])."""
    Lp = _f64(Lp)
    D, M = Lp.shape
    out_phys = _f64(out_phys)
    res = np.array(in_phys, dtype=np.float64, copy=True)
    rc = _load().oracle_lplustimes(M, D, G, Z, layout_in, layout_out, _p(Lp), _p(out_phys), _p(res))
    if rc != 0:
        raise ValueError("oracle_lplustimes: invalid arguments")
    return res


def ltimes_sample(L: np.ndarray, x_phys: np.ndarray, G: int, Z: int, layout_in: int,
                  idx: np.ndarray) -> np.ndarray:
    """out at canonical (m, g, z) rows of idx (shape (S, 3))."""
    L = _f64(L)
    x_phys = _f64(x_phys)
    M, D = L.shape
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    vals = np.empty(idx.shape[0], dtype=np.float64)
    rc = _load().oracle_ltimes_sample(M, D, G, Z, layout_in, _p(L), _p(x_phys), idx.shape[0], _p(idx), _p(vals))
    if rc != 0:
        raise ValueError("oracle_ltimes_sample: index out of range")
    return vals


class MLPParams:
    """FP64 parameters of the F -> H -> H -> 1 ReLU network."""

    NAMES = ("W1", "b1", "W2", "b2", "w3", "b3")

    def __init__(self, W1, b1, W2, b2, w3, b3):
        self.W1, self.b1, self.W2 = _f64(W1), _f64(b1), _f64(W2)
        self.b2, self.w3, self.b3 = _f64(b2), _f64(w3), _f64(np.reshape(b3, (1,)))

    @property
    def F(self):
        return self.W1.shape[1]

    @property
    def H(self):
        return self.W1.shape[0]

    def tensors(self):
        return [self.W1, self.b1, self.W2, self.b2, self.w3, self.b3]

    def flat(self) -> np.ndarray:
        return np.concatenate([t.ravel() for t in self.tensors()])

    @classmethod
    def from_flat(cls, v: np.ndarray, F: int, H: int) -> "MLPParams":
        sizes = [H * F, H, H * H, H, H, 1]
        parts, o = [], 0
        for s in sizes:
            parts.append(v[o:o + s])
            o += s
        return cls(parts[0].reshape(H, F), parts[1], parts[2].reshape(H, H), parts[3], parts[4], parts[5])


def mlp_forward(p: MLPParams, X: np.ndarray):
    X = _f64(X)
    B = X.shape[0]
    y = np.empty(B)
    h1 = np.empty((B, p.H))
    h2 = np.empty((B, p.H))
    _load().oracle_mlp_forward(p.F, p.H, B, *[_p(t) for t in p.tensors()], _p(X), _p(y), _p(h1), _p(h2))
    return y, h1, h2


def mlp_loss_grad(p: MLPParams, X: np.ndarray, t: np.ndarray):
    """(loss, MLPParams of gradients)."""
    X = _f64(X)
    t = _f64(t)
    g = MLPParams(np.empty_like(p.W1), np.empty_like(p.b1), np.empty_like(p.W2),
                  np.empty_like(p.b2), np.empty_like(p.w3), np.empty(1))
    loss = _load().oracle_mlp_loss_grad(p.F, p.H, X.shape[0], *[_p(a) for a in p.tensors()],
                                        _p(X), _p(t), *[_p(a) for a in g.tensors()])
    return loss, g


def adam(theta: np.ndarray, grad: np.ndarray, m: np.ndarray, v: np.ndarray, step: int,
         lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """In-place Adam step on float64 flat vectors."""
    for a in (theta, grad, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    _load().oracle_adam(theta.size, _p(theta), _p(grad), _p(m), _p(v), step, lr, beta1, beta2, eps)


def eigen_bench(n: int, repeat: int) -> np.ndarray:
    out = np.empty((n, n))
    _load().oracle_eigen_bench(n, repeat, _p(out))
    return out


def eigen_recurrence(M0: np.ndarray, repeat: int, c: float = 5e-5) -> np.ndarray:
    """Batched M_{k+1} = Ones + c (M_k + M_k M_k) from starts M0 [batch][n][n] (Sec. 5, Listing eigen1)."""
    M0 = np.ascontiguousarray(M0, dtype=np.float64)
    b, n, _ = M0.shape
    out = np.empty_like(M0)
    _load().oracle_eigen_recurrence(b, n, repeat, c, _p(M0), _p(out))
    return out


def eigen_start(n: int) -> np.ndarray:
    """The listing's start M_0(i, j) = i + n j."""
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return (i + n * j).astype(np.float64)


def mass(B1: np.ndarray, op: np.ndarray, x: np.ndarray, dim: int, nthreads: int = 1) -> np.ndarray:
    """Mass operator of tensor-product elements: y_e = B^T diag(op_e) B x_e,
    B the dim-fold Kronecker product of B1 (Q x D).  x: [ne][D^dim], op:
    [ne][Q^dim] (first index fastest within an element); returns y like x."""
    B1 = _f64(B1)
    Q, D = B1.shape
    x = _f64(x).reshape(-1, D ** dim)
    op = _f64(op).reshape(-1, Q ** dim)
    assert x.shape[0] == op.shape[0]
    y = np.empty_like(x)
    rc = _load().oracle_mass(dim, D, Q, x.shape[0], _p(B1), _p(op), _p(x), _p(y), nthreads)
    if rc != 0:
        raise ValueError("oracle_mass: invalid arguments")
    return y
