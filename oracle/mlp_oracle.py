"""CPU reference of the selector network (numpy, float64).

TEST INFRASTRUCTURE ONLY (the GPU gradient check compares against it).

Network 48 -> 64 -> 64 -> 1, ReLU, logit output, weighted mean binary
cross-entropy.  Parameters packed as W1[48][64], b1[64], W2[64][64], b2[64],
w3[64], b3.  With quantise=True the BF16 rounding points of the GPU kernels
are applied (round to nearest even on the float32 value):
    X_q, W1_q, W2_q, H1_q = bf16(relu(A1)), dH2_q, dH1_q
everything else in float64.  With quantise=False it is the plain network,
whose gradient the tests check against central differences.
"""
from __future__ import annotations

import numpy as np

NF, NH = 48, 64
P_W1 = 0
P_B1 = NF * NH
P_W2 = P_B1 + NH
P_B2 = P_W2 + NH * NH
P_W3 = P_B2 + NH
P_B3 = P_W3 + NH
NPARAM = P_B3 + 1


def bf16(x):
    """round float32 values to the nearest bfloat16 (ties to even), as float64"""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[P_W1:P_B1].reshape(NF, NH), p[P_B1:P_W2], p[P_W2:P_B2].reshape(NH, NH), p[P_B2:P_W3],
            p[P_W3:P_B3], p[P_B3])


def forward(p, X, quantise=True):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    q = bf16 if quantise else (lambda a: np.asarray(a, dtype=np.float64))
    Xq = q(X)
    A1 = Xq @ q(W1) + b1
    H1 = np.maximum(A1, 0.0)
    H1q = q(H1)
    A2 = H1q @ q(W2) + b2
    H2 = np.maximum(A2, 0.0)
    z = H2 @ w3 + b3
    return dict(Xq=Xq, A1=A1, H1q=H1q, A2=A2, H2=H2, z=z)


def loss_and_grad(p, X, y, wgt=None, quantise=True):
    """weighted mean BCE of the logits and its gradient w.r.t. the packed parameters"""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    q = bf16 if quantise else (lambda a: np.asarray(a, dtype=np.float64))
    y = np.asarray(y, dtype=np.float64)
    wgt = np.ones_like(y) if wgt is None else np.asarray(wgt, dtype=np.float64)
    f = forward(p, X, quantise)
    z = f["z"]
    wsum = wgt.sum()
    loss = np.sum(wgt * (np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z))))) / wsum
    s = 1.0 / (1.0 + np.exp(-z))
    dz = (s - y) * wgt / wsum
    g = np.zeros(NPARAM)
    g[P_W3:P_B3] = f["H2"].T @ dz
    g[P_B3] = dz.sum()
    dH2 = np.outer(dz, w3) * (f["A2"] > 0)
    g[P_B2:P_W3] = dH2.sum(axis=0)
    dH2q = q(dH2)
    g[P_W2:P_B2] = (f["H1q"].T @ dH2q).ravel()
    dH1 = (dH2q @ q(W2).T) * (f["A1"] > 0)
    g[P_B1:P_W2] = dH1.sum(axis=0)
    dH1q = q(dH1)
    g[P_W1:P_B1] = (f["Xq"].T @ dH1q).ravel()
    return loss, g
