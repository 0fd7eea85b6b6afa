"""CPU oracle of the learned warm start (test infrastructure only).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
CPU-baseline leg may import this module; the product path never does and
shares no code with it.

The paper has no learned component: it starts every solve from a given point
(x^{0,0}, y^{0,0}) (Algorithm 1 takes it as input; Section 5 uses zero).  The
warm-start network maps the data (c, b) of one member of a parameterised QP
family to a starting point (x0, y0).  Its definition, restated here in the
plainest form:

  * normalisation: per feature f of v = [c; b], u_f = (v_f - mean_f) * scale_f
    with mean/scale from the training inputs (scale = 1 / population std, 1
    where the std is below 1e-8); targets t = [x*; y*] likewise with
    t_f = (y_f - omean_f) * oinv_f and the prediction
    y_f = omean_f + ostd_f * o_f;
  * h_0 = u P' with a fixed random projection P (d x (n+m));
  * h_j = relu(h_{j-1} W_j' + b_j), j = 1..depth (width w);
  * o = h_depth W_out' + b_out;
  * loss = mean over samples and features of (o - t)^2;
  * Adam (Kingma & Ba 2015, Algorithm 1) with bias correction.

Precision: the network stores weights and activations in bfloat16 and
accumulates in float32.  With mimic=True this oracle rounds to bfloat16 at
exactly the points where the GPU path stores bfloat16 (u, h_j, the bf16 weight
copies, the gradients fed to the weight-gradient and input-gradient products)
and to float32 where it stores float32 (o, the gradients before rounding, the
normalisation vectors), but every sum is formed in float64.  With mimic=False
it is plain float64 throughout (used for the finite-difference pins).
"""
import numpy as np


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even) via float32, returned as float64."""
    x = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    bits = x.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    bits = ((bits + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return bits.view(np.float32).astype(np.float64)


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


# --------------------------------------------------------------------------
# normalisation
# --------------------------------------------------------------------------
def _mean_std(V):
    mean = V.mean(axis=0)
    std = np.sqrt(((V - mean) ** 2).mean(axis=0))
    std = np.where(std < 1e-8, 1.0, std)
    return mean, std


def fit_normalization(C, B, X, Y):
    """Per-feature statistics of inputs [C | B] and targets [X | Y] (rows are
    samples).  Returns float32 arrays in_mean, in_scale, out_mean, out_std,
    out_inv."""
    mi, si = _mean_std(np.hstack([C, B]))
    mo, so = _mean_std(np.hstack([X, Y]))
    return dict(in_mean=mi.astype(np.float32), in_scale=(1.0 / si).astype(np.float32),
                out_mean=mo.astype(np.float32), out_std=so.astype(np.float32),
                out_inv=(1.0 / so).astype(np.float32))


def prep_input(C, B, norm, mimic=True):
    """u = (v - mean) * scale, in float32 arithmetic then rounded to bfloat16."""
    V = np.hstack([C, B])
    if not mimic:
        return (V - norm["in_mean"]) * norm["in_scale"]
    d = np.float32(V.astype(np.float32)) - norm["in_mean"]
    return bf16_round(d.astype(np.float32) * norm["in_scale"])


def prep_target(X, Y, norm, mimic=True):
    V = np.hstack([X, Y])
    if not mimic:
        return (V - norm["out_mean"]) * norm["out_inv"]
    d = V.astype(np.float32) - norm["out_mean"]
    return f32(d.astype(np.float32) * norm["out_inv"])


def prediction(O, norm, n):
    """Split o back into (x0, y0) in the problem's units."""
    V = norm["out_mean"].astype(np.float64) + norm["out_std"].astype(np.float64) * O
    return V[:, :n], V[:, n:]


# --------------------------------------------------------------------------
# forward / backward
# --------------------------------------------------------------------------
def forward(layers, proj, U, mimic=True):
    """layers: list of (W, b) float32 arrays, hidden layers then the output
    layer.  Returns (H, O): H[0] = h_0 ... H[depth] and the output o."""
    rb = bf16_round if mimic else (lambda a: a)
    h = rb(U @ rb(proj).T)
    H = [h]
    for W, b in layers[:-1]:
        h = rb(np.maximum(h @ rb(W).T + b, 0.0))
        H.append(h)
    W, b = layers[-1]
    O = h @ rb(W).T + b
    return H, (f32(O) if mimic else O)


def loss_and_grads(layers, proj, U, T, mimic=True):
    """Mean squared error and its gradient for every (W, b) of `layers`."""
    rb = bf16_round if mimic else (lambda a: a)
    rf = f32 if mimic else (lambda a: a)
    H, O = forward(layers, proj, U, mimic)
    S, F = T.shape
    R = O - T
    loss = float(np.mean(R * R))
    depth = len(layers) - 1
    grads = [None] * len(layers)
    # float32 on the device: g = (o - t) * fl32(2 / (S F))
    dZ = f32(f32(R) * np.float32(2.0 / (S * F))) if mimic else (2.0 / (S * F)) * R
    for j in range(depth, -1, -1):                 # layer j maps H[j] -> next
        W, _ = layers[j]
        dZb = rb(dZ)
        gW = dZb.T @ H[j]
        gb = dZ.sum(axis=0)
        grads[j] = (gW, gb)
        if j > 0:
            dH = dZb @ rb(W)
            dZ = rf(np.where(H[j] > 0.0, dH, 0.0))
    return loss, grads


# --------------------------------------------------------------------------
# Adam
# --------------------------------------------------------------------------
def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of parameter p with gradient g, moments m, v, at step
    t >= 1.  Returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def affine_permutation(count, epoch, seed):
    """Visit order of the training samples in one epoch: i -> (a*i + s) mod count
    with a coprime to count, from a 64-bit mix of (seed, epoch)."""
    z = _mix64((seed * 0x9E3779B97F4A7C15 + epoch * 0xD1B54A32D192ED03) & 0xFFFFFFFFFFFFFFFF)
    a = int(z % count) | 1
    while np.gcd(a, count) != 1:
        a += 2
    a %= count
    if a == 0:
        a = 1
    s = int((z >> 32) % count)
    return (a * np.arange(count, dtype=np.int64) + s) % count


def _mix64(z):
    """SplitMix64 finaliser (Steele, Lea & Flood 2014)."""
    M = 0xFFFFFFFFFFFFFFFF
    z = (z + 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def train(layers, proj, C, B, X, Y, norm, epochs, batch, lr, seed, beta1=0.9, beta2=0.999, eps=1e-8,
          mimic=True):
    """Minibatch Adam over the samples in affine-permutation order (the last
    partial batch of an epoch is dropped).  Returns (layers, losses per
    epoch)."""
    U = prep_input(C, B, norm, mimic)
    T = prep_target(X, Y, norm, mimic)
    H0 = bf16_round(U @ bf16_round(proj).T) if mimic else U @ proj.T
    count = U.shape[0]
    layers = [(W.astype(np.float64), b.astype(np.float64)) for W, b in layers]
    mom = [(np.zeros_like(W), np.zeros_like(b), np.zeros_like(W), np.zeros_like(b)) for W, b in layers]
    eye = np.eye(proj.shape[0])
    losses, t = [], 0
    for e in range(epochs):
        order = affine_permutation(count, e, seed)
        tot, nb = 0.0, 0
        for s0 in range(0, count - batch + 1, batch):
            idx = order[s0:s0 + batch]
            loss, grads = loss_and_grads(layers, eye, H0[idx], T[idx], mimic)
            t += 1
            new = []
            for (W, b), (gW, gb), (mW, mb, vW, vb) in zip(layers, grads, mom):
                W, mW, vW = adam_step(W, gW, mW, vW, t, lr, beta1, beta2, eps)
                b, mb, vb = adam_step(b, gb, mb, vb, t, lr, beta1, beta2, eps)
                new.append(((W, b), (mW, mb, vW, vb)))
            layers = [p for p, _ in new]
            mom = [q for _, q in new]
            tot += loss
            nb += 1
        losses.append(tot / max(nb, 1))
    return layers, losses
