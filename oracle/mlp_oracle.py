"""FP64 CPU oracle of the learned proposal -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import this module.  It shares no
code with the CUDA path.  Everything is plain numpy in FP64.

What the learned proposal computes (the learned form of the data-driven predictor of Section 3.2):

* For every region R and case, the data-driven predictor of Section 3.2 gives coefficients c_R of its
  prediction in the stored-snapshot basis: y_R = Y_R c_R.
* A small network maps the features of the region and case to a correction of those coefficients.  The
  features are the source position relative to the region centroid (divided by the domain extent), the
  normalised source frequency and c_R itself.  The proposal is c_R + net(features), and the guess is
  Y_R (c_R + net(features)).
* The network is trained to the best coefficients in the same basis, c*_R = argmin ||Y_R c - e_R^it||,
  where e^it is the correction that the solve then finds.  Its regression target is c*_R - c_R.

Readings (the paper states the data-driven predictor, and the network form is set by the workload):
  L1  network 64 -> 256 -> 256 -> 32, GELU (erf form) after the first two layers, linear output.  The 36
      used inputs are zero-padded to 64.
  L2  inputs x[0:3] = (source position - region centroid) / L, with L the largest edge of the domain's
      bounding box; x[3] = (f0 - 5) / 3; x[4:36] = asinh(c_R) in age order (entry k belongs to the pair whose
      output is e^{it-1-k}); missing pairs are 0.  asinh keeps the inputs bounded where nearly collinear
      snapshots give least-squares coefficients of 1e6 and more.
  L3  the network predicts the correction c*_R - c_R (residual form), so an untrained (zero-output) network
      reproduces the data-driven predictor.
  L4  targets c*_R use the same column-drop rule as the predictor (R9), applied to the columns of Y_R.  A
      sample whose correction c*_R - c_R has a non-finite entry or one above TARGET_CLIP in magnitude gets the
      target 0 (no correction): such coefficient jumps come from nearly collinear columns, where
      coefficient space says little about the prediction Y_R c.
  L5  loss = mean over samples and the 32 outputs of the squared error; Adam with bias correction
      (lr 1e-3, beta = 0.9 / 0.999, eps = 1e-8).
  L6  residual-space loss (the quantity the acceptance test decides on): the relative error of a case's
      corrected guess of the correction, sum over regions R of ||Y_R (c_R + d_R) - e_R||^2 divided by ||e||^2
      of the whole case at that step (each region's share is one sample; a per-region ||e_R||^2 would blow up
      where the wave has not arrived yet and e_R is nearly zero).  d_R is the network output in age order.  With Y_R's
      columns in age order, MGS (drop rule R9) gives P with orthonormal kept columns and R = P^T Y_R (upper
      triangular); then ||Y_R (c_R + d) - e_R||^2 = ||R (c_R + d) - P^T e_R||^2 + ||(I - P P^T) e_R||^2 (up
      to the dropped columns' parts outside span(P), below tau of their norms), so a sample's share is
      ||W d - w||^2 + const with W = R / ||e|| and w = (P^T e_R - R c_R) / ||e||.  A sample stores W (upper
      triangle, row by row) and w; no target clipping is needed, since directions Y_R leaves undetermined
      carry no weight.  Loss = mean over samples of ||W d - w||^2.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from .fem_oracle import mgs_upper

LAYERS = (64, 256, 256, 32)
N_COEF = 32
N_USED = 4 + N_COEF
F0_CENTER, F0_SCALE = 5.0, 3.0
TARGET_CLIP = 100.0


# ---------------------------------------------------------------------------------------------------------
# Parameters: one flat FP64 vector in the order W1 [256][64], b1 [256], W2 [256][256], b2 [256],
# W3 [32][256], b3 [32] (the same order the GPU library uses for its parameter and gradient buffers).
# ---------------------------------------------------------------------------------------------------------

def param_shapes():
    out = []
    for i in range(3):
        out.append((LAYERS[i + 1], LAYERS[i]))
        out.append((LAYERS[i + 1],))
    return out


def n_params():
    return sum(int(np.prod(s)) for s in param_shapes())


def unpack(theta):
    res, o = [], 0
    for s in param_shapes():
        k = int(np.prod(s))
        res.append(theta[o:o + k].reshape(s))
        o += k
    return res


def pack(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


# ---------------------------------------------------------------------------------------------------------
# Network (L1)
# ---------------------------------------------------------------------------------------------------------

def gelu(x):
    """GELU(x) = x * Phi(x), Phi the standard normal CDF, Phi(x) = (1 + erf(x / sqrt 2)) / 2."""
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    """d/dx [x Phi(x)] = Phi(x) + x phi(x), phi the standard normal density."""
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(theta, X):
    """X [B][64] -> (out [B][32], cache).  Layer l: Z_l = A_{l-1} W_l^T + b_l; A_l = GELU(Z_l) for l < 3."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    Z1 = X @ W1.T + b1
    A1 = gelu(Z1)
    Z2 = A1 @ W2.T + b2
    A2 = gelu(Z2)
    out = A2 @ W3.T + b3
    return out, (X, Z1, A1, Z2, A2)


def loss(theta, X, T):
    out, _ = forward(theta, X)
    return float(np.mean((out - T) ** 2))


def loss_and_grad(theta, X, T):
    """Mean squared error over all B x 32 outputs and its gradient (reverse mode, layer by layer)."""
    out, cache = forward(theta, X)
    B = X.shape[0]
    diff = out - T
    L = float(np.mean(diff ** 2))
    d3 = 2.0 * diff / (B * out.shape[1])          # dL/dout
    return L, backprop(theta, cache, d3)


def backprop(theta, cache, d3):
    """Gradient of a loss with respect to the parameters, given dL/dout = d3 [B][32]."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X0, Z1, A1, Z2, A2 = cache
    gW3 = d3.T @ A2
    gb3 = d3.sum(axis=0)
    d2 = (d3 @ W3) * gelu_grad(Z2)                 # dL/dZ2
    gW2 = d2.T @ A1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * gelu_grad(Z1)                 # dL/dZ1
    gW1 = d1.T @ X0
    gb1 = d1.sum(axis=0)
    return pack([gW1, gb1, gW2, gb2, gW3, gb3])


# ---------------------------------------------------------------------------------------------------------
# Residual-space loss (L6)
# ---------------------------------------------------------------------------------------------------------
N_TRI = N_COEF * (N_COEF + 1) // 2          # packed upper triangle of W
N_RES = N_TRI + N_COEF                      # one residual-space sample: W then w


def pack_residual(W, w):
    """[W upper triangle row by row (i <= j), w] as one vector of N_RES values."""
    iu = np.triu_indices(N_COEF)
    return np.concatenate([W[iu], w])


def unpack_residual(S):
    """Inverse of pack_residual for a [B][N_RES] array: (W [B][32][32], w [B][32])."""
    S = np.atleast_2d(S)
    B = S.shape[0]
    W = np.zeros((B, N_COEF, N_COEF))
    iu = np.triu_indices(N_COEF)
    W[:, iu[0], iu[1]] = S[:, :N_TRI]
    return W, S[:, N_TRI:].copy()


def residual_sample(Y, e, c, tau=1e-6, norm2=None):
    """(W [32][32], w [32]) of one sample (L6).  Y [rows][n]: the region's stored outputs y_a = e^{it-n+a}
    (oldest first), e the region's part of the correction the solve found, c [n] the predictor's coefficients
    (slot order), norm2 the case's normalisation ||e||^2 over all regions (default: the region's own).  Everything is
    returned in age order (index k belongs to the pair whose output is e^{it-1-k})."""
    n = Y.shape[1]
    W = np.zeros((N_COEF, N_COEF))
    w = np.zeros(N_COEF)
    ne = float(np.linalg.norm(e)) if norm2 is None else math.sqrt(float(norm2))
    if n == 0 or ne == 0.0:
        return W, w
    Ya = Y[:, ::-1]                      # age order
    ca = np.asarray(c, dtype=np.float64)[::-1]
    _, P, _ = mgs_upper(Ya, tau)
    R = P.T @ Ya
    W[:n, :n] = R / ne
    w[:n] = (P.T @ e - R @ ca) / ne
    return W, w


def loss_residual(theta, X, S):
    """L6 loss: mean over the samples of ||W d - w||^2, d = net(x)."""
    out, _ = forward(theta, X)
    W, w = unpack_residual(S)
    r = np.einsum("bij,bj->bi", W, out) - w
    return float(np.mean(np.sum(r * r, axis=1)))


def loss_and_grad_residual(theta, X, S):
    """L6 loss and its gradient: dL/dd_b = 2 W_b^T (W_b d_b - w_b) / B, then the same reverse pass."""
    out, cache = forward(theta, X)
    W, w = unpack_residual(S)
    B = X.shape[0]
    r = np.einsum("bij,bj->bi", W, out) - w
    L = float(np.mean(np.sum(r * r, axis=1)))
    d3 = 2.0 * np.einsum("bij,bi->bj", W, r) / B
    return L, backprop(theta, cache, d3)


def train_residual(theta, X, S, batches, lr=1e-3):
    """Adam on the L6 loss over the given minibatch index arrays; returns (theta, losses before each update)."""
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    losses = []
    for t, idx in enumerate(batches, start=1):
        L, g = loss_and_grad_residual(theta, X[idx], S[idx])
        losses.append(L)
        theta, m, v = adam_step(theta, g, m, v, t, lr)
    return theta, losses


def adam_step(theta, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update with bias correction (t = 1 for the first step).  Returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def train(theta, X, T, batches, lr=1e-3):
    """Adam over the given list of minibatch index arrays; returns (theta, losses before each update)."""
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    losses = []
    for t, idx in enumerate(batches, start=1):
        L, g = loss_and_grad(theta, X[idx], T[idx])
        losses.append(L)
        theta, m, v = adam_step(theta, g, m, v, t, lr)
    return theta, losses


# ---------------------------------------------------------------------------------------------------------
# Features and targets (L2-L4)
# ---------------------------------------------------------------------------------------------------------

def domain_extent(xyz):
    return float((xyz.max(axis=0) - xyz.min(axis=0)).max())


def region_centroids(xyz, region_of_node, n_regions):
    """Mean position of the nodes of each region."""
    C = np.zeros((n_regions, 3))
    for R in range(n_regions):
        C[R] = xyz[region_of_node == R].mean(axis=0)
    return C


def features(src_pos, centroid, extent, f0, coef_slot_order):
    """Input vector [64] of one (region, case).  coef_slot_order: the predictor's coefficients, column a
    of Y being e^{it-n+a} (oldest first); they enter in age order (newest first)."""
    x = np.zeros(LAYERS[0])
    x[0:3] = (np.asarray(src_pos) - np.asarray(centroid)) / extent
    x[3] = (f0 - F0_CENTER) / F0_SCALE
    n = len(coef_slot_order)
    for a in range(n):
        c = coef_slot_order[a]
        x[4 + (n - 1 - a)] = math.asinh(c) if math.isfinite(c) else 0.0
    return x


def target(best_slot_order, pred_slot_order):
    """Regression target in age order: c* - c, or zero when that correction is not finite or exceeds
    TARGET_CLIP in magnitude (L4)."""
    d = np.asarray(best_slot_order, dtype=np.float64) - np.asarray(pred_slot_order, dtype=np.float64)
    if d.size and (not np.all(np.isfinite(d)) or np.abs(d).max() > TARGET_CLIP):
        d = np.zeros_like(d)
    return to_age_order(d)


def best_coefficients(Y, e, tau=1e-6):
    """c* = argmin ||Y c - e|| by modified Gram-Schmidt on the columns of Y (dropped columns get 0)."""
    if Y.shape[1] == 0:
        return np.zeros(0)
    U, P, _ = mgs_upper(Y, tau)
    return U @ (P.T @ e)


def to_age_order(coef_slot_order, n_out=N_COEF):
    out = np.zeros(n_out)
    n = len(coef_slot_order)
    for a in range(n):
        out[n - 1 - a] = coef_slot_order[a]
    return out


def from_age_order(coef_age, n):
    return np.array([coef_age[n - 1 - a] for a in range(n)])


def step_samples_residual(sim, src_pos, centroids, extent, f0, tau=1e-6):
    """Residual-space samples (L6) of the step `sim` has just taken: per region (features at prediction time,
    packed (W, w)).  Returns (X [R][64], S [R][N_RES])."""
    n = sim.last_npairs
    R_all = sim.n_regions
    X = np.zeros((R_all, LAYERS[0]))
    S = np.zeros((R_all, N_RES))
    W = sim.last_W
    if n > 0:
        Y = np.stack(sim.E_hist[-(n + 1):-1], axis=1)
        e = sim.E_hist[-1]
        D = float(e @ e)
    for R in range(R_all):
        c = W[R, :n] if n > 0 else np.zeros(0)
        X[R] = features(src_pos, centroids[R], extent, f0, c)
        if n > 0:
            idx = np.nonzero(sim.region_of_dof == R)[0]
            S[R] = pack_residual(*residual_sample(Y[idx], e[idx], c, tau, norm2=D))
    return X, S


def plain_error2(Y, e, W, n, region_of_dof, n_regions):
    """D = sum over regions of ||Y_R c_R - e_R||^2: the plain guess's squared error of the correction."""
    D = 0.0
    for R in range(n_regions):
        idx = np.nonzero(region_of_dof == R)[0]
        r = Y[idx] @ W[R, :n] - e[idx]
        D += float(r @ r)
    return D


def step_samples(sim, src_pos, centroids, extent, f0, tau=1e-6):
    """Training samples of the step `sim` has just taken (CaseSimulator with the data-driven predictor):
    per region, (features at prediction time, target c*_R - c_R in age order).  Returns (X [R][64],
    T [R][32]); regions are all of the simulator's regions, in order."""
    n = sim.last_npairs
    R_all = sim.n_regions
    X = np.zeros((R_all, LAYERS[0]))
    T = np.zeros((R_all, N_COEF))
    W = sim.last_W
    if n > 0:
        Y = np.stack(sim.E_hist[-(n + 1):-1], axis=1)
        e = sim.E_hist[-1]
    for R in range(R_all):
        c = W[R, :n] if n > 0 else np.zeros(0)
        X[R] = features(src_pos, centroids[R], extent, f0, c)
        if n > 0:
            idx = np.nonzero(sim.region_of_dof == R)[0]
            cs = best_coefficients(Y[idx], e[idx], tau)
            T[R] = target(cs, c)
    return X, T
