"""VQE optimisation on the GPU MPS, plain and surrogate-assisted.

The paper's VQE demonstration (Sec. V.B) evaluates the energy of an ansatz
for a sweep of parameter values. Here an optimiser drives the parameters:

* ``MPSEnergy``: batched E(theta) through the C ABI (every call counts its
  MPS evaluations).
* ``param_shift``: exact gradient dE/dtheta_j = [E(theta + pi/2 e_j) -
  E(theta - pi/2 e_j)] / 2 for exp(-i theta sigma / 2) gates, 2P + 1
  evaluations (the centre included).
* ``plain_adam``: Adam on the parameter-shift gradient.
* ``surrogate_adam``: the same exact-gradient Adam steps, each followed by
  steps proposed from the MLP surrogate's input gradient (no MPS evaluation
  to propose), every proposal verified by one MPS evaluation and kept only if
  its MPS energy is lower. Every MPS-evaluated point (proposals and the 2P
  parameter-shift points) joins the surrogate's training data, and the
  surrogate is fine-tuned on recent points. The MPS is therefore both the
  fallback and the arbiter: the reported energies are all MPS energies.
"""
import json
import time

import numpy as np
import torch

from . import inputs, tnmps


class MPSEnergy:
    """E(theta) for rows of theta on the GPU MPS; counts evaluations."""

    def __init__(self, n, chi, eps, circuit, n_params, terms, dtype="c128", batch=640,
                 device="cuda:0"):
        self.P = int(n_params)
        self.batch = int(batch)
        self.device = torch.device(device)
        self.m = tnmps.MPSBatch(n, chi, self.batch, dtype=dtype, max_params=self.P, eps=eps,
                                device=self.device)
        self.ps = tnmps.PauliSum(n, terms)
        self.gates = tnmps.gate_array(circuit)
        self.th = torch.zeros((self.batch, self.P), dtype=torch.float64, device=self.device)
        self.e = torch.empty(self.batch, dtype=torch.float64, device=self.device)
        self.evals = 0

    def __call__(self, thetas):
        thetas = np.atleast_2d(np.asarray(thetas, dtype=np.float64))
        out = np.empty(thetas.shape[0])
        for s in range(0, thetas.shape[0], self.batch):
            chunk = thetas[s:s + self.batch]
            k = chunk.shape[0]
            buf = np.empty((self.batch, self.P))
            buf[:k] = chunk
            buf[k:] = chunk[-1]
            self.th.copy_(torch.from_numpy(buf))
            self.m.reset()
            self.m.apply_circuit_dev(self.gates, self.th)
            self.m.expect_dev(self.ps, self.e)
            out[s:s + k] = self.e[:k].cpu().numpy()
        self.m.check()
        self.evals += thetas.shape[0]
        return out


def param_shift(energy, theta):
    """(E(theta), exact gradient) with 2P + 1 MPS evaluations."""
    P = theta.size
    rows = np.repeat(theta[None, :], 2 * P + 1, axis=0)
    idx = np.arange(P)
    rows[1 + idx, idx] += 0.5 * np.pi
    rows[1 + P + idx, idx] -= 0.5 * np.pi
    e = energy(rows)
    return e[0], 0.5 * (e[1:P + 1] - e[P + 1:]), rows, e


class Adam:
    def __init__(self, P, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(P)
        self.v = np.zeros(P)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def propose(self, theta, g, lr=None):
        t = self.t + 1
        m = self.b1 * self.m + (1 - self.b1) * g
        v = self.b2 * self.v + (1 - self.b2) * g * g
        step = (lr or self.lr) * (m / (1 - self.b1 ** t)) / (np.sqrt(v / (1 - self.b2 ** t)) + self.eps)
        return theta - step, (m, v, t)

    def commit(self, state):
        self.m, self.v, self.t = state


def plain_adam(energy, theta0, lr, max_evals, target=None):
    """Adam on exact parameter-shift gradients. Returns (history, best)."""
    theta = np.array(theta0, dtype=np.float64)
    opt = Adam(theta.size, lr)
    hist, best = [], (np.inf, theta.copy())
    while energy.evals < max_evals:
        e0, g, _, _ = param_shift(energy, theta)
        if e0 < best[0]:
            best = (e0, theta.copy())
        hist.append((energy.evals, float(best[0])))
        if target is not None and best[0] <= target:
            break
        theta, st = opt.propose(theta, g)
        opt.commit(st)
    return hist, best


def wrap(theta):
    """The energy is 2 pi periodic in every parameter: the surrogate sees
    angles in [-pi, pi)."""
    return (np.asarray(theta) + np.pi) % (2 * np.pi) - np.pi


def _init_params(d, w, rng):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    parts = [rng.uniform(-1, 1, (w, d)) / np.sqrt(d), np.zeros(w),
             rng.uniform(-1, 1, (w, w)) / np.sqrt(w), np.zeros(w),
             rng.uniform(-1, 1, w) / np.sqrt(w), np.zeros(1)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


class Surrogate:
    """Standardised MLP model of E(theta) trained on MPS data."""

    def __init__(self, P, width=256, max_batch=4096, device="cuda:0", seed=0):
        self.P = P
        self.device = torch.device(device)
        self.net = tnmps.Surrogate(P, width, max_batch=max_batch, device=self.device)
        self.net.set_params(_init_params(P, width, np.random.default_rng(seed)))
        self.mu, self.sd = 0.0, 1.0
        self.X = np.zeros((0, P))
        self.Y = np.zeros(0)
        self.max_batch = max_batch

    def add(self, X, Y):
        self.X = np.concatenate([self.X, wrap(X)])
        self.Y = np.concatenate([self.Y, Y])

    def fit(self, epochs, lr, batch=4096, recent=None, rng=None, restandardise=False):
        rng = rng or np.random.default_rng(0)
        X, Y = (self.X, self.Y) if recent is None else (self.X[-recent:], self.Y[-recent:])
        if restandardise:
            self.mu, self.sd = float(self.Y.mean()), float(self.Y.std() + 1e-12)
        batch = min(batch, self.max_batch, X.shape[0])
        Xd = torch.tensor(X, dtype=torch.float32, device=self.device)
        Yd = torch.tensor((Y - self.mu) / self.sd, dtype=torch.float32, device=self.device)
        loss = None
        for _ in range(epochs):
            perm = torch.from_numpy(rng.permutation(X.shape[0])).to(self.device)
            for s in range(0, X.shape[0] - batch + 1, batch):
                sel = perm[s:s + batch]
                loss = self.net.train_step(Xd[sel], Yd[sel], lr)
        return float(loss.item()) * self.sd ** 2 if loss is not None else None

    def predict(self, X):
        x = torch.tensor(wrap(np.atleast_2d(X)), dtype=torch.float32, device=self.device)
        return self.net.forward(x).double().cpu().numpy() * self.sd + self.mu

    def grad(self, theta):
        x = torch.tensor(wrap(theta)[None, :], dtype=torch.float32, device=self.device)
        _, _, gx = self.net.backward(x, None, want_params=False, want_x=True)
        return gx[0].double().cpu().numpy() * self.sd


def surrogate_adam(energy, sur, theta0, lr, max_evals, target=None, sur_steps=8,
                   finetune_epochs=2, finetune_lr=3e-4, recent=20000, rng=None):
    """Exact-gradient Adam backbone plus surrogate extrapolation.

    Every iteration takes one Adam step on the exact parameter-shift
    gradient (2P + 1 MPS evaluations, which also become training data), then
    up to ``sur_steps`` further steps proposed from the surrogate's gradient
    with the backbone's moment estimates (not committed), each verified by
    one MPS evaluation and kept only while the MPS energy decreases. The
    surrogate is fine-tuned on the most recent points after each iteration."""
    rng = rng or np.random.default_rng(0)
    theta = np.array(theta0, dtype=np.float64)
    opt = Adam(theta.size, lr)
    hist = []
    best = np.inf
    stats = {"iterations": 0, "proposals": 0, "accepted": 0}
    while energy.evals < max_evals:
        e0, g, rows, es = param_shift(energy, theta)
        sur.add(rows, es)
        best = min(best, e0)
        hist.append((energy.evals, best))
        if target is not None and best <= target:
            break
        theta, st = opt.propose(theta, g)
        opt.commit(st)
        e = float(energy(theta[None])[0])
        sur.add(theta[None], np.array([e]))
        best = min(best, e)
        hist.append((energy.evals, best))
        for _ in range(sur_steps):
            cand, _ = opt.propose(theta, sur.grad(theta))
            ec = float(energy(cand[None])[0])
            sur.add(cand[None], np.array([ec]))
            stats["proposals"] += 1
            if not ec < e:
                break
            theta, e = cand, ec
            stats["accepted"] += 1
            best = min(best, e)
            hist.append((energy.evals, best))
        stats["iterations"] += 1
        sur.fit(finetune_epochs, finetune_lr, recent=recent, rng=rng)
    return hist, (best, theta), stats


def evals_to(hist, target):
    for ev, e in hist:
        if e <= target:
            return ev
    return None


def main():
    import argparse
    ap = argparse.ArgumentParser(description="surrogate-assisted vs plain VQE on the MPS")
    ap.add_argument("--n-data", type=int, default=100000)
    ap.add_argument("--budget", type=int, default=200000)
    ap.add_argument("--lr", type=float, default=0.02)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    wl = inputs.workload("heis40")
    P = wl["n_params"]
    t0 = time.time()
    gen = MPSEnergy(wl["n"], wl["chi_max"], wl["eps"], wl["circuit"], P, wl["terms"], "c64", 2048)
    rng = np.random.default_rng(4000 + a.seed)
    X = rng.uniform(-np.pi, np.pi, (a.n_data, P))
    Y = gen(X)
    t_data = time.time() - t0
    sur = Surrogate(P)
    sur.add(X, Y)
    t1 = time.time()
    train_mse = sur.fit(a.epochs, 1e-3, restandardise=True)
    t_train = time.time() - t1
    theta0 = rng.uniform(-np.pi, np.pi, P)
    plain = MPSEnergy(wl["n"], wl["chi_max"], wl["eps"], wl["circuit"], P, wl["terms"], "c128", 641)
    hp, bp = plain_adam(plain, theta0, a.lr, a.budget)
    verifier = MPSEnergy(wl["n"], wl["chi_max"], wl["eps"], wl["circuit"], P, wl["terms"], "c128", 641)
    hs, bs, st = surrogate_adam(verifier, sur, theta0, a.lr, a.budget)
    e_star = min(bp[0], bs[0])
    target = e_star + 1e-4
    out = {"workload": "heis40: n=40, 4 layers Ry/Rz + CNOT ladder (320 params), chi 64, "
                       "cutoff 1e-10, Heisenberg 157 terms",
           "n_data": a.n_data, "data_s": t_data, "train_s": t_train, "train_mse": train_mse,
           "E0": float(plain(theta0[None])[0]), "E_star": e_star, "target": target,
           "plain_best": bp[0], "surrogate_best": bs[0],
           "plain_evals_to_target": evals_to(hp, target),
           "surrogate_evals_to_target": evals_to(hs, target),
           "surrogate_evals_to_plain_best": evals_to(hs, bp[0]),
           "plain_evals_to_plain_best": evals_to(hp, bp[0]),
           "plain_evals": hp[-1][0], "surrogate_evals": hs[-1][0], "surrogate_stats": st}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
