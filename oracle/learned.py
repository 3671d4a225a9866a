"""The learned correction of the fast-diagonalisation patch inverse, in plain
NumPy FP64 (test infrastructure: it checks the CUDA forward/backward kernels).

Model (a two-layer perceptron, our design; the paper has none):
  features  x = log a_c - mean_c log a_c over the 2^d cells of a patch
  hidden    h = tanh(W1 x + b1)
  output    o = W2 h + b2,  U[i, q] = o[i * R + q] (i < m^d, q < R), s[q] = o[m^d R + q]
  solve     d = theta Ahat^{-1} r  +  U diag(s) U^T r   (reference units, coefficient
            w = a/abar; theta = min(1, 1.8 / max_c w_c), the FD damping)
Loss per sample: ||d - d_exact||^2 / ||d_exact||^2, averaged over the batch,
with d_exact the exact solve with the normalised patch matrix; DFD holds the
damped FD term theta Ahat^{-1} r.

Pinned (tests/test_oracle_varcoef.py): the analytic gradients against finite
differences of the loss; the output layout and the loss's units by the
full-rank eigen-correction (loss exactly zero) and by rank-r truncations
(per eigenvector residual the loss is zero for a kept mode and s_q^2/||DEX||^2
for a dropped one).
"""
import numpy as np


def forward(params, X):
    W1, b1, W2, b2 = params
    H = np.tanh(X @ W1.T + b1)
    return H, H @ W2.T + b2


def split(O, nint, rank):
    U = O[:, :nint * rank].reshape(-1, nint, rank)
    s = O[:, nint * rank:nint * rank + rank]
    return U, s


def correction(O, R, nint, rank):
    U, s = split(O, nint, rank)
    t = np.einsum("nir,ni->nr", U, R)
    return np.einsum("nir,nr->ni", U, s * t)


def loss(params, X, R, DFD, DEX, rank):
    _, O = forward(params, X)
    nint = R.shape[1]
    E = DFD + correction(O, R, nint, rank) - DEX
    return np.mean(np.sum(E ** 2, axis=1) / np.sum(DEX ** 2, axis=1))


def loss_and_grads(params, X, R, DFD, DEX, rank):
    """Analytic gradients (chain rule through the rank-R correction and the
    two layers)."""
    W1, b1, W2, b2 = params
    N, nint = R.shape
    H, O = forward(params, X)
    U, s = split(O, nint, rank)
    t = np.einsum("nir,ni->nr", U, R)                 # U^T r
    w = s * t
    E = DFD + np.einsum("nir,nr->ni", U, w) - DEX
    scale = 2.0 / (N * np.sum(DEX ** 2, axis=1))      # d loss / d E = scale * E
    G = scale[:, None] * E                            # [N, nint]
    gUt = np.einsum("nir,ni->nr", U, G)               # U^T g
    dU = np.einsum("ni,nr->nir", G, w) + np.einsum("ni,nr->nir", R, s * gUt)
    ds = t * gUt
    dO = np.concatenate([dU.reshape(N, nint * rank), ds], axis=1)
    dW2 = dO.T @ H
    db2 = dO.sum(axis=0)
    dH = (dO @ W2) * (1.0 - H ** 2)
    dW1 = dH.T @ X
    db1 = dH.sum(axis=0)
    L = np.mean(np.sum(E ** 2, axis=1) / np.sum(DEX ** 2, axis=1))
    return L, (dW1, db1, dW2, db2)
