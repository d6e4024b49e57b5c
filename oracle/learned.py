"""Learned correction stage of the FGMRES solve (the learned form; the paper's
Sec. 4 solver has no such stage, it is an extra smoothing step on top of the
Alg. 2 preconditioner).  Test infrastructure only: plain FP64 numpy, no code
shared with the CUDA library.

Per Q2 node a of a 2D mesh, with its 3x3 lattice patch N(a) (slot s = 3*(dj+1) +
(di+1), absent neighbours outside the mesh):

  x_{s,k} = r'[dof_k(N_s(a))] / sigma_in[class(dof)]   k = v_x, v_y, u_x, u_y, p
            (0 for an absent neighbour, and for p at a node that carries no p)
  rho_a   = sqrt(sum of the 45 squares / 45)
  f_a     = [x / rho_a (45 values, slot-major), one-hot of the lattice parity
             (i odd) + 2 (j odd) (4), flags solid / v fixed / u fixed / interface (4)]

In 3D the patch is the 3x3x3 neighbourhood (slot s = 9*(dk+1) + 3*(dj+1) + (di+1)),
k runs over v_x, v_y, v_z, u_x, u_y, u_z, p (189 values), the parity one-hot has 8
entries ((i odd) + 2 (j odd) + 4 (k odd)), so f_a has 201 inputs and y_a 7 outputs.
  y_a     = W3^T gelu(W2^T gelu(W1^T f_a + b1) + b2) + b3,   gelu(x) = x Phi(x)
  c[dof_k(a)] = y_{a,k} rho_a sigma_out[class(dof)]   (0 on fixed rows, at rho_a = 0
             and for p at a node without p)

so the correction is positively homogeneous of degree 1 in r'.  Classes are the
five DOF blocks m, s_v, s_u, f_v, f_p of the monolithic system.  Weights are
stored in bfloat16 (round to nearest even); every product and sum here is FP64.

Inside FGMRES (right preconditioning, Saad Alg. 9.6), with z_j = P^-1 v_j:
  q = A z_j,  r' = v_j - q,  c = MLP(r'),  t = A c;
  if ||r' - t|| < tau ||r'||:  z_j <- z_j + c,  w = q + t   (accepted; tau in (0, 1])
  else:                        w = q                        (the plain preconditioner)
The stage never changes what FGMRES converges to, only the search space.

Training (the learned stage's own loss, not in the paper): for a pair
(r', e = A^-1 r'), the error e - c of the correction measured in the residual
norm that the accept test compares, L = ||A (e - c)||^2 / ||r'||^2
= ||r' - A c||^2 / ||r'||^2, minimised by backpropagation and AdamW
(Loshchilov & Hutter 2019) on FP32 master weights whose bfloat16 rounding is
what the forward pass uses.  The targets() helper gives e in the network's
output units (diagnostics).
"""
from __future__ import annotations

import math
import struct

import numpy as np
from scipy.special import erf

N_HIDDEN = 64


def layout(dim: int):
    """(n_in, n_out, n_patch, n_slots, n_comp, n_parity) of the stage in `dim` dimensions."""
    comp, slots, par = 2 * dim + 1, 3 ** dim, 2 ** dim
    return slots * comp + par + 4, comp, slots * comp, slots, comp, par


def shapes(dim: int):
    n_in, n_out = layout(dim)[:2]
    return [("W1", (n_in, N_HIDDEN)), ("b1", (N_HIDDEN,)), ("W2", (N_HIDDEN, N_HIDDEN)), ("b2", (N_HIDDEN,)),
            ("W3", (N_HIDDEN, n_out)), ("b3", (n_out,))]


def n_params(dim: int) -> int:
    return sum(int(np.prod(s)) for _, s in shapes(dim))


N_IN, N_OUT, N_PATCH = layout(2)[:3]
SHAPES = shapes(2)
N_PARAMS = n_params(2)
N_PARAMS_3D = n_params(3)
MAGIC = b"FSIMLP01"

FLAG_SOLID, FLAG_VFIX, FLAG_UFIX, FLAG_IFACE, FLAG_IODD, FLAG_JODD, FLAG_PFIX, FLAG_KODD = 1, 2, 4, 8, 16, 32, 64, 128


def dim_of_params(params) -> int:
    n = len(np.asarray(params).reshape(-1))
    for d in (2, 3):
        if n == n_params(d):
            return d
    raise ValueError("parameter count of neither the 2D nor the 3D stage")


def dim_of_patch(patch) -> int:
    w = np.asarray(patch).shape[1]
    if w not in (9, 27):
        raise ValueError("patch width must be 9 (2D) or 27 (3D)")
    return 2 if w == 9 else 3


# ------------------------------------------------------------------ bfloat16
def bf16_bits(x) -> np.ndarray:
    """float32 -> bfloat16 bit patterns, round to nearest, ties to even."""
    u = np.array(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    return ((u + 0x7FFF + lsb) >> 16).astype(np.uint16)


def bf16_value(bits) -> np.ndarray:
    """bfloat16 bit patterns -> exact float64 values."""
    b = np.asarray(bits, np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)


def unflatten(params) -> dict:
    p = np.asarray(params, np.float64)
    out, k = {}, 0
    for name, shape in shapes(dim_of_params(p)):
        size = int(np.prod(shape))
        out[name] = p[k:k + size].reshape(shape)
        k += size
    return out


def flatten(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SHAPES])   # order only


# ------------------------------------------------------------------ weights file
def read_weights(path: str):
    """Weights file: 8-byte magic, int32 n_in n_hidden n_out reserved, float32
    sigma_in[5] sigma_out[5], then the bfloat16 parameters W1 b1 W2 b2 W3 b3
    (row-major, W_l maps layer input (rows) to output (columns)), little endian."""
    with open(path, "rb") as f:
        raw = f.read()
    if raw[:8] != MAGIC:
        raise ValueError("not an MLP weights file")
    n_in, n_h, n_out, _ = struct.unpack_from("<4i", raw, 8)
    dims = {layout(d)[:2]: d for d in (2, 3)}
    if n_h != N_HIDDEN or (n_in, n_out) not in dims:
        raise ValueError("unexpected MLP shape")
    scales = np.frombuffer(raw, "<f4", 10, 24).astype(np.float64)
    bits = np.frombuffer(raw, "<u2", n_params(dims[(n_in, n_out)]), 64)
    return bits.copy(), scales[:5].copy(), scales[5:].copy()


# ------------------------------------------------------------------ features
def dof_class(dofs, offsets) -> np.ndarray:
    """Class 0..4 (m, s_v, s_u, f_v, f_p) of each DOF index (monolithic order)."""
    return np.searchsorted(np.asarray(offsets[1:5]), np.asarray(dofs), side="right")


def node_dofs(node_dof, dim: int = 2) -> np.ndarray:
    """[n_nodes, 2 dim + 1] DOF of (v components, u components, p) at each node, -1 where absent."""
    nd = np.asarray(node_dof)
    cols = [nd[:, 0] + i for i in range(dim)] + [nd[:, 1] + i for i in range(dim)] + [nd[:, 2]]
    return np.stack(cols, axis=1)


def features(rp, node_dof, patch, offsets, sigma_in):
    """(F [n_nodes, n_in], rho [n_nodes]) for residual r' (the definition above); the
    dimension follows from the patch width."""
    dim = dim_of_patch(patch)
    n_in, _, n_patch, n_slots, n_comp, n_par = layout(dim)
    rp = np.asarray(rp, np.float64)
    sig = np.asarray(sigma_in, np.float64)
    D = node_dofs(node_dof, dim)                            # [n_nodes, n_comp]
    scaled = np.zeros(D.shape)
    ok = D >= 0
    scaled[ok] = rp[D[ok]] / sig[dof_class(D[ok], offsets)]
    pt = np.asarray(patch)
    X = np.zeros((pt.shape[0], n_slots, n_comp))
    has = pt >= 0
    X[has] = scaled[pt[has]]
    X = X.reshape(-1, n_patch)
    rho = np.sqrt(np.sum(X * X, axis=1) / n_patch)
    F = np.zeros((X.shape[0], n_in))
    nz = rho > 0
    F[nz, :n_patch] = X[nz] / rho[nz, None]
    fl = np.asarray(node_dof)[:, 3]
    par = ((fl & FLAG_IODD) != 0).astype(int) + 2 * ((fl & FLAG_JODD) != 0).astype(int)
    if dim == 3:
        par = par + 4 * ((fl & FLAG_KODD) != 0).astype(int)
    F[np.arange(len(par)), n_patch + par] = 1.0
    for k, bit in enumerate((FLAG_SOLID, FLAG_VFIX, FLAG_UFIX, FLAG_IFACE)):
        F[:, n_patch + n_par + k] = ((fl & bit) != 0).astype(np.float64)
    return F, rho


def output_mask(node_dof, dim: int = 2) -> np.ndarray:
    """[n_nodes, 2 dim + 1]: 1 where the node's output k is a free DOF."""
    nd = np.asarray(node_dof)
    fl = nd[:, 3]
    M = np.ones((nd.shape[0], 2 * dim + 1))
    M[(fl & FLAG_VFIX) != 0, 0:dim] = 0.0
    M[(fl & FLAG_UFIX) != 0, dim:2 * dim] = 0.0
    M[(nd[:, 2] < 0) | ((fl & FLAG_PFIX) != 0), 2 * dim] = 0.0
    return M


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def mlp_forward(params, F, keep=False):
    """y = W3^T gelu(W2^T gelu(W1^T f + b1) + b2) + b3 for each row f of F."""
    P = unflatten(params)
    h1 = F @ P["W1"] + P["b1"]
    a1 = gelu(h1)
    h2 = a1 @ P["W2"] + P["b2"]
    a2 = gelu(h2)
    y = a2 @ P["W3"] + P["b3"]
    if keep:
        return y, (F, h1, a1, h2, a2)
    return y


def correction(rp, node_dof, patch, offsets, bits, sigma_in, sigma_out):
    """c = MLP(r') scattered to the monolithic vector (the definition above)."""
    dim = dim_of_patch(patch)
    F, rho = features(rp, node_dof, patch, offsets, sigma_in)
    y = mlp_forward(bf16_value(bits), F)
    D = node_dofs(node_dof, dim)
    M = output_mask(node_dof, dim) * (rho > 0)[:, None]
    c = np.zeros(np.asarray(rp).shape[0])
    ok = (M > 0) & (D >= 0)
    sig = np.asarray(sigma_out, np.float64)
    vals = y * rho[:, None]
    c[D[ok]] = vals[ok] * sig[dof_class(D[ok], offsets)]
    return c


def targets(e, node_dof, offsets, rho, sigma_out, dim: int = 2):
    """(Y, M): y*_{a,k} = e[dof_k(a)] / (rho_a sigma_out[class]) and its mask."""
    e = np.asarray(e, np.float64)
    D = node_dofs(node_dof, dim)
    M = output_mask(node_dof, dim) * (np.asarray(rho) > 0)[:, None]
    Y = np.zeros(D.shape)
    ok = (M > 0) & (D >= 0)
    sig = np.asarray(sigma_out, np.float64)
    den = np.broadcast_to(np.asarray(rho, np.float64)[:, None], D.shape)[ok] * sig[dof_class(D[ok], offsets)]
    Y[ok] = e[D[ok]] / den
    return Y, M


# ------------------------------------------------------------------ training
def mlp_backward(params, cache, dy) -> np.ndarray:
    """dL/dparams of the forward pass in `cache` for output gradients dy [n_nodes, n_out]."""
    P = unflatten(params)
    X, h1, a1, h2, a2 = cache
    g = {"W3": a2.T @ dy, "b3": dy.sum(0)}
    dh2 = (dy @ P["W3"].T) * gelu_grad(h2)
    g["W2"] = a1.T @ dh2
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ P["W2"].T) * gelu_grad(h1)
    g["W1"] = X.T @ dh1
    g["b1"] = dh1.sum(0)
    return flatten(g)


def residual_loss_and_grad(params, rp, A, node_dof, patch, offsets, sigma_in, sigma_out):
    """L = ||r' - A c||^2 / ||r'||^2 for c = MLP(r') with the parameters as given
    (FP64), and dL/dparams: dL/dc = -2 A^T (r' - A c) / ||r'||^2, then
    dL/dy_{a,k} = dL/dc[dof_k(a)] rho_a sigma_out[class] on free outputs, then
    backpropagation through the layers."""
    rp = np.asarray(rp, np.float64)
    dim = dim_of_patch(patch)
    F, rho = features(rp, node_dof, patch, offsets, sigma_in)
    y, cache = mlp_forward(params, F, keep=True)
    D = node_dofs(node_dof, dim)
    M = output_mask(node_dof, dim) * (rho > 0)[:, None]
    ok = (M > 0) & (D >= 0)
    sig = np.asarray(sigma_out, np.float64)
    scale = np.zeros(D.shape)
    scale[ok] = np.broadcast_to(rho[:, None], D.shape)[ok] * sig[dof_class(D[ok], offsets)]
    c = np.zeros(rp.shape[0])
    c[D[ok]] = y[ok] * scale[ok]
    res = rp - A @ c
    nr = float(rp @ rp)
    L = float(res @ res) / nr
    gc = -2.0 * (A.T @ res) / nr
    dy = np.zeros(D.shape)
    dy[ok] = gc[D[ok]] * scale[ok]
    return L, mlp_backward(params, cache, dy)


def adamw_step(w, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
    """One AdamW update (decoupled weight decay) at step t >= 1; returns (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    w = w - lr * (mhat / (np.sqrt(vhat) + eps) + weight_decay * w)
    return w, m, v


class LearnedStage:
    """Callable r' -> c for the oracle FGMRES (see fgmres(..., correct=...))."""

    def __init__(self, node_dof, patch, offsets, bits, sigma_in, sigma_out):
        self.node_dof, self.patch, self.offsets = node_dof, patch, np.asarray(offsets)
        self.bits, self.sigma_in, self.sigma_out = bits, sigma_in, sigma_out

    @classmethod
    def from_file(cls, path, node_dof, patch, offsets):
        bits, si, so = read_weights(path)
        return cls(node_dof, patch, offsets, bits, si, so)

    def __call__(self, rp):
        return correction(rp, self.node_dof, self.patch, self.offsets, self.bits, self.sigma_in, self.sigma_out)
