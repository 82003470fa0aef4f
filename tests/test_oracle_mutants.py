"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/oracle.c (a dropped term, a
wrong constant, a transposed operand, a wrong index or an off-by-one loop),
builds it with the oracle's own flags, binds it in place of the real library
and runs a set of independent pins -- closed forms, special cases that reduce
to a library routine, and identities -- written here against numpy, not
against the oracle.  Every mutant must fail at least one pin of its group,
and the unmodified oracle must pass them all.  The mistakes are planted in
the oracle only, on the CPU."""
import contextlib
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import synth

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")


@contextlib.contextmanager
def bound(path):
    """The oracle module calls the library at `path` inside the block."""
    prev = oracle._lib
    oracle._lib = oracle._bind(ctypes.CDLL(path))
    try:
        yield
    finally:
        oracle._lib = prev


def build_mutant(tmp_path, name, old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, (name, old)
    src = tmp_path / f"{name}.c"
    src.write_text(text.replace(old, new))
    lib = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", *oracle.CFLAGS, "-o", str(lib), str(src), "-lm"], check=True)
    return str(lib)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


# ---------------------------------------------------------------------------
# Pins (True when the pin holds), each against numpy or a closed form
# ---------------------------------------------------------------------------

def chain_pins():
    pins = {}
    n, T = 3, 5
    pins["A = 0 gives I"] = np.array_equal(oracle.update_chain(np.zeros((1, n, n)), T)[0], np.eye(n))
    X = oracle.update_chain(np.eye(n)[None], T)[0]
    pins["A = I gives (1 + 1/(N T))^T I"] = rel(X, (1 + 1 / (n * T)) ** T * np.eye(n)) <= 1e-14
    A = synth.chain_inputs_np(0x51, 3, 4)
    ref = np.stack([np.linalg.matrix_power(np.eye(4) + a / (4 * 7), 7) for a in A])
    pins["(I + A/(N T))^T by matrix powers"] = rel(oracle.update_chain(A, 7), ref) <= 1e-12
    Ac = synth.chain_inputs_np(0x52, 2, 5, layout=1)
    Xc = oracle.update_chain(Ac, 6, layout=1)
    refc = np.stack([np.linalg.matrix_power(np.eye(5) + a.T / 30, 6) for a in Ac])
    pins["column-major storage"] = rel(Xc.transpose(0, 2, 1), refc) <= 1e-12
    return pins


def ltimes_pins():
    pins = {}
    M, D, G, Z = 3, 5, 2, 4
    L, x = synth.ltimes_inputs_np(0x53, M, D, G, Z)
    ref = np.einsum("md,dgz->mgz", L, x)
    ok = True
    for lin in range(6):
        for lout in range(6):
            out = oracle.ltimes(L, synth.to_layout(x, lin).ravel(), G, Z, lin, lout)
            ok = ok and rel(synth.from_layout(out, lout, (M, G, Z)), ref) <= 1e-13
    pins["every order pair equals numpy's contraction"] = ok
    sel = np.zeros((M, D))
    sel[np.arange(M), np.arange(M)] = 1.0
    out = oracle.ltimes(sel, x.ravel(), G, Z, 0, 0).reshape(M, G, Z)
    pins["a selector L copies in's first rows"] = np.array_equal(out, x[:M])
    return pins


def lplustimes_pins():
    pins = {}
    M, D, G, Z = 3, 4, 2, 5
    Lp = synth.uniform_np(0x54, 0, D * M).reshape(D, M)
    y = synth.uniform_np(0x55, 0, M * G * Z).reshape(M, G, Z)
    base = synth.uniform_np(0x56, 0, D * G * Z).reshape(D, G, Z)
    got = oracle.lplustimes(Lp, y.ravel(), base.ravel(), G, Z, 0, 0).reshape(D, G, Z)
    pins["in + Lp out by numpy"] = rel(got, base + np.einsum("dm,mgz->dgz", Lp, y)) <= 1e-13
    L = Lp.T.copy()
    x = synth.uniform_np(0x57, 0, D * G * Z).reshape(D, G, Z)
    lhs = float(np.sum(oracle.ltimes(L, x.ravel(), G, Z, 0, 0) * y.ravel()))
    rhs = float(np.sum(x.ravel() * oracle.lplustimes(Lp, y.ravel(), np.zeros(D * G * Z), G, Z, 0, 0)))
    pins["adjoint identity"] = abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    return pins


def mass_pins():
    pins = {}
    D = Q = 3
    ne = 4
    x = synth.uniform_np(0x58, 0, ne * D * D).reshape(ne, D * D)
    op = synth.uniform_np(0x59, 0, ne * Q * Q).reshape(ne, Q * Q) + 2.0
    y = oracle.mass(np.eye(3), op, x, 2)
    pins["identity basis scales x by op"] = np.array_equal(y, op * x)
    D, Q = 2, 3
    B1 = synth.uniform_np(0x5A, 0, Q * D).reshape(Q, D)
    x = synth.uniform_np(0x5B, 0, 2 * D * D).reshape(2, D * D)
    op = synth.uniform_np(0x5C, 0, 2 * Q * Q).reshape(2, Q * Q)
    B = np.kron(B1, B1)   # quadrature multi-index (k2, k1) against dof (j2, j1): first index fastest
    ref = np.stack([B.T @ (o * (B @ v)) for o, v in zip(op, x)])
    pins["B^T diag(op) B x with numpy's Kronecker product"] = rel(oracle.mass(B1, op, x, 2), ref) <= 1e-13
    return pins


def eigen_pins():
    pins = {}
    M0 = oracle.eigen_start(4)
    M1 = 1.0 + 5e-5 * (M0 + M0 @ M0)
    pins["one step from the listing's start"] = rel(oracle.eigen_bench(4, 1), M1) <= 1e-15
    starts = synth.uniform_np(0x5D, 0, 2 * 9).reshape(2, 3, 3)
    got = oracle.eigen_recurrence(starts, 2, 0.25)
    ref = []
    for m in starts:
        for _ in range(2):
            m = 1.0 + 0.25 * (m + m @ m)
        ref.append(m)
    pins["batched recurrence, two steps"] = rel(got, np.stack(ref)) <= 1e-14
    return pins


def mlp_pins():
    pins = {}
    F, H, B = 3, 4, 6
    rng = np.random.default_rng(11)
    p = oracle.MLPParams(rng.uniform(-1, 1, (H, F)), rng.uniform(-1, 1, H), rng.uniform(-1, 1, (H, H)),
                         rng.uniform(-1, 1, H), rng.uniform(-1, 1, H), rng.uniform(-1, 1, 1))
    X = rng.uniform(-1, 1, (B, F))
    t = rng.uniform(-1, 1, B)
    _, g = oracle.mlp_loss_grad(p, X, t)
    theta, gflat = p.flat(), g.flat()
    ok = True
    for i in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += 1e-6
        tm[i] -= 1e-6
        lp, _ = oracle.mlp_loss_grad(oracle.MLPParams.from_flat(tp, F, H), X, t)
        lm, _ = oracle.mlp_loss_grad(oracle.MLPParams.from_flat(tm, F, H), X, t)
        ok = ok and abs((lp - lm) / 2e-6 - gflat[i]) <= 1e-6 * max(1.0, abs(gflat[i]))
    pins["central finite differences"] = ok
    th = np.array([1.0, -2.0, 0.5])
    g0 = np.array([0.3, -0.7, 2.0])
    m, v = np.zeros(3), np.zeros(3)
    oracle.adam(th, g0, m, v, 1, lr=0.01)
    # first step with bias correction: m_hat = g, v_hat = g^2, so theta moves by lr * g / (|g| + eps)
    pins["first Adam step moves each parameter by lr"] = rel(th, [1.0 - 0.01 * 0.3 / (0.3 + 1e-8),
                                                                 -2.0 + 0.01 * 0.7 / (0.7 + 1e-8),
                                                                 0.5 - 0.01 * 2.0 / (2.0 + 1e-8)]) <= 1e-12
    return pins


GROUPS = {"chain": chain_pins, "ltimes": ltimes_pins, "lplustimes": lplustimes_pins, "mass": mass_pins,
          "eigen": eigen_pins, "mlp": mlp_pins}

MUTANTS = [
    # (name, group, text in oracle.c, planted mistake)
    ("chain_drops_x", "chain", "x[i * n + j] = x[i * n + j] + c * p[i * n + j];", "x[i * n + j] = c * p[i * n + j];"),
    ("chain_wrong_c", "chain", "const double c = 1.0 / ((double)n * (double)steps);",
     "const double c = 1.0 / ((double)steps);"),
    ("chain_transposed_a", "chain", "sum = sum + x[i * n + l] * a[l * n + j];",
     "sum = sum + x[i * n + l] * a[j * n + l];"),
    ("chain_one_step_short", "chain", "for (int k = 0; k < steps; ++k) {", "for (int k = 1; k < steps; ++k) {"),
    ("chain_ignores_layout", "chain", "a[r * n + s] = (layout == 0) ? A[r * n + s] : A[s * n + r];",
     "a[r * n + s] = A[r * n + s];"),
    ("ltimes_wrong_order_1", "ltimes", "case 1: return (x * ez + z) * eg + g;   /* X Z G */",
     "case 1: return (x * eg + g) * ez + z;   /* X Z G */"),
    ("ltimes_wrong_order_4", "ltimes", "case 4: return (z * ex + x) * eg + g;   /* Z X G */",
     "case 4: return (z * eg + g) * ex + x;   /* Z X G */"),
    ("ltimes_transposed_l", "ltimes", "sum = sum + j->L[(int64_t)m * j->D + d] *",
     "sum = sum + j->L[(int64_t)d * j->M + m] *"),
    ("ltimes_skips_first_d", "ltimes", "for (int d = 0; d < j->D; ++d)\n                    sum = sum + j->L",
     "for (int d = 1; d < j->D; ++d)\n                    sum = sum + j->L"),
    ("lplustimes_overwrites", "lplustimes", "in[o] = in[o] + sum;", "in[o] = sum;"),
    ("lplustimes_transposed_lp", "lplustimes", "sum = sum + Lp[(int64_t)d * M + m] *",
     "sum = sum + Lp[(int64_t)m * D + d] *"),
    ("mass_drops_op", "mass", "u[k] = op[k] * s;", "u[k] = s;"),
    ("mass_swapped_kronecker", "mass", "v = v * j->B1[(kr % Q) * D + (jr % D)];",
     "v = v * j->B1[(jr % Q) * D + (kr % D)];"),
    ("mass_back_uses_x", "mass", "for (int k = 0; k < nq; ++k) s = s + B[(size_t)k * nd + jj] * u[k];",
     "for (int k = 0; k < nq; ++k) s = s + B[(size_t)k * nd + jj] * op[k];"),
    ("eigen_drops_m", "eigen", "for (int i = 0; i < n * n; ++i) m[i] = 1.0 + 5e-5 * (m[i] + q[i]);",
     "for (int i = 0; i < n * n; ++i) m[i] = 1.0 + 5e-5 * q[i];"),
    ("eigen_transposed_start", "eigen", "m[i * n + j] = (double)(i + n * j);", "m[i * n + j] = (double)(n * i + j);"),
    ("mlp_loss_half_gradient", "mlp", "double dy = 2.0 * r / (double)B;", "double dy = r / (double)B;"),
    ("mlp_relu_passes_negative", "mlp", "d1[i] = (z1[i] > 0.0) ? s : 0.0;", "d1[i] = s;"),
    ("adam_no_bias_correction", "mlp", "const double mh = m[i] / c1;", "const double mh = m[i];"),
]


@pytest.mark.parametrize("group", sorted(GROUPS))
def test_unmodified_oracle_passes_every_pin(group):
    pins = GROUPS[group]()
    assert all(pins.values()), {k: v for k, v in pins.items() if not v}


@pytest.mark.parametrize("name,group,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, name, group, old, new):
    lib = build_mutant(tmp_path, name, old, new)
    with bound(lib):
        pins = GROUPS[group]()
    failed = [k for k, v in pins.items() if not v]
    assert failed, f"no pin of group {group} catches {name}"


# ---------------------------------------------------------------------------
# The key contract (oracle/keys.py): hand-assembled bytes and the variant rule
# ---------------------------------------------------------------------------

def keys_pins(K):
    u16 = lambda v: int(v).to_bytes(2, "little")
    u32 = lambda v: int(v).to_bytes(4, "little")
    pins = {}
    want = (u16(1) + bytes([0, 1, 0, 0]) + u16(12) + u16(0) + u16(0) +
            u32(1) + u32(21) + u32(0) + u32(0) + u32(2))
    pins["chain key, column-major, NO_AOT"] = K.canonical_key(1, 0, n=12, layout_a=1, tile=(1, 21, 0, 0),
                                                              flags=2) == want
    want = (u16(2) + bytes([1, 3, 5, 0]) + u16(0) + u16(36) + u16(96) +
            u32(1) + u32(128) + u32(320) + u32(6685700) + u32(0))
    pins["LTimes key ignores n, keeps both orders"] = K.canonical_key(2, 1, n=7, layout_a=3, layout_b=5, m=36, d=96,
                                                                      tile=(1, 128, 320, 6685700)) == want
    want = u16(3) + bytes([1, 0, 0, 0]) + u16(40) + u16(0) + u16(0) + u32(8) + u32(2) + u32(0) + u32(0) + u32(0)
    pins["grouped key zeroes the layout"] = K.canonical_key(3, 1, n=40, layout_a=1, tile=(8, 2, 0, 0)) == want
    want = u16(1) + bytes([0, 0, 0, 0]) + u16(5) + u16(0) * 2 + u32(0) * 4 + u32(1)
    pins["GENERIC drops the tile"] = K.canonical_key(1, 0, n=5, tile=(1, 32, 0, 0), flags=1) == want
    pins["unknown flag bits are dropped"] = (K.canonical_key(1, 0, n=5, tile=(1, 32, 0, 0), flags=0x4) ==
                                             K.canonical_key(1, 0, n=5, tile=(1, 32, 0, 0)))
    pins["variant rule"] = (K.expected_variant(1, 1, 32, True) == 1 and K.expected_variant(1, 0, 16, True) == 1 and
                            K.expected_variant(1, 0, 16, False) == 2 and K.expected_variant(1, 0, 5, True) == 2 and
                            K.expected_variant(1, 0, 8, True, flags=2) == 2 and
                            K.expected_variant(1, 0, 8, True, flags=1) == 0 and
                            K.expected_variant(1, 2, 16, True) == 2 and K.expected_variant(3, 0, 8, True) == 2)
    return pins


KEY_MUTANTS = [
    ("keys_swapped_orders", "layout_a, layout_b, 0, n, m, d, *tile", "layout_b, layout_a, 0, n, m, d, *tile"),
    ("keys_grouped_keeps_layout", "            layout_a = 0\n", "            pass\n"),
    ("keys_generic_keeps_tile", "        tile = (0, 0, 0, 0)\n", "        pass\n"),
    ("keys_all_flags_kept", "*tile, flags & KEY_FLAGS)", "*tile, flags)"),
    ("keys_aot_set_without_32", "AOT_SIZES = (4, 8, 16, 32)", "AOT_SIZES = (4, 8, 16)"),
    ("keys_aot_for_explicit_tiles", "\n            and tile_left_to_library and", "\n            and"),
    ("keys_ltimes_keeps_n", "    elif kernel in (K_LTIMES, K_LPLUSTIMES):\n        n = 0\n",
     "    elif kernel in (K_LTIMES, K_LPLUSTIMES):\n        pass\n"),
]


def keys_module(text):
    import types
    mod = types.ModuleType("keys_copy")
    exec(compile(text, "keys_copy.py", "exec"), mod.__dict__)
    return mod


def test_unmodified_keys_pass_every_pin():
    from oracle import keys as K
    pins = keys_pins(K)
    assert all(pins.values()), {k: v for k, v in pins.items() if not v}


@pytest.mark.parametrize("name,old,new", KEY_MUTANTS, ids=[m[0] for m in KEY_MUTANTS])
def test_planted_key_mistake_fails_a_pin(name, old, new):
    from oracle import keys as K
    text = open(K.__file__).read()
    assert text.count(old) == 1, name
    pins = keys_pins(keys_module(text.replace(old, new)))
    assert [k for k, v in pins.items() if not v], f"no key pin catches {name}"
