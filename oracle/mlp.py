"""FP64 oracle of the detection-schedule network (16 -> 64 -> 64 -> 2, ReLU).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy, double precision.  The
GPU computes its products on BF16 operands with FP32 accumulation; ``bf16=True`` rounds
every product operand to BF16 (round to nearest even) the same way, so that the two
differ only by the FP32 accumulation.  The analytic gradient is pinned by central finite
differences of the forward pass (tests/test_oracle_mlp.py).

Parameter layout (flat): W1[64][16], b1[64], W2[64][64], b2[64], W3[2][64], b3[2].
Loss: mean over rows and outputs of w (y_hat - y)^2, w = 4 where y_hat > y, else 1.
"""
import numpy as np

IN, H, OUT = 16, 64, 2
SHAPES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (OUT, H)), ("b3", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)
OVERSHOOT = 4.0


def unpack(p):
    out, k = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(p[k:k + n], np.float64).reshape(shp)
        k += n
    return out


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _q(x, on):
    return bf16(x) if on else np.asarray(x, np.float64)


def forward(p, X, bf=True, keep=False):
    P = unpack(p)
    X = np.asarray(X, np.float64)
    a1 = _q(X, bf) @ _q(P["W1"], bf).T + P["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = _q(h1, bf) @ _q(P["W2"], bf).T + P["b2"]
    h2 = np.maximum(a2, 0.0)
    out = _q(h2, bf) @ _q(P["W3"], bf).T + P["b3"]
    if keep:
        return out, (X, h1, h2)
    return out


def loss(p, X, Y, bf=True):
    e = forward(p, X, bf) - np.asarray(Y, np.float64)
    w = np.where(e > 0, OVERSHOOT, 1.0)
    return float(np.mean(w * e * e))


def loss_grad(p, X, Y, bf=True):
    """Loss and its gradient by the chain rule (transposed products of the forward)."""
    P = unpack(p)
    out, (X, h1, h2) = forward(p, X, bf, keep=True)
    Y = np.asarray(Y, np.float64)
    e = out - Y
    w = np.where(e > 0, OVERSHOOT, 1.0)
    n = e.size
    L = float(np.mean(w * e * e))
    d_out = 2.0 * w * e / n
    g = {}
    g["W3"] = _q(d_out, bf).T @ _q(h2, bf)
    g["b3"] = d_out.sum(axis=0)
    d_h2 = (_q(d_out, bf) @ _q(P["W3"], bf)) * (h2 > 0)
    g["W2"] = _q(d_h2, bf).T @ _q(h1, bf)
    g["b2"] = d_h2.sum(axis=0)
    d_h1 = (_q(d_h2, bf) @ _q(P["W2"], bf)) * (h1 > 0)
    g["W1"] = _q(d_h1, bf).T @ _q(X, bf)
    g["b1"] = d_h1.sum(axis=0)
    grad = np.concatenate([g[name].ravel() for name, _ in SHAPES])
    return L, grad


def blocks():
    """(name, slice) of each parameter block in the flat layout."""
    out, k = [], 0
    for name, shp in SHAPES:
        m = int(np.prod(shp))
        out.append((name, slice(k, k + m)))
        k += m
    return out


def gradient_tolerance(g_ref):
    """Per-element tolerance of a BF16-operand gradient against g_ref (this oracle with
    bf=True): one BF16 ulp of the element (2^-7 of it), plus 2^-14 of the largest entry
    of its block for entries that cancel to near zero.  Both sides round the same
    operands to BF16; they differ only in the precision of the sums and intermediates
    (FP32 against FP64), which moves an operand across a BF16 rounding boundary only
    rarely, and then changes one term of a sum by one BF16 ulp."""
    g_ref = np.asarray(g_ref, np.float64)
    tol = np.empty_like(g_ref)
    for _, sl in blocks():
        tol[sl] = 2.0 ** -7 * np.abs(g_ref[sl]) + 2.0 ** -14 * np.max(np.abs(g_ref[sl]))
    return tol

