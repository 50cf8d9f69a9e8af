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
    """E(theta) for rows of theta on the GPU MPS; counts evaluations. Calls
    with fewer rows than ``small`` run on a second context of ``small``
    states, so a single proposal does not pay for a full parameter-shift
    batch."""

    def __init__(self, n, chi, eps, circuit, n_params, terms, dtype="c128", batch=640,
                 device="cuda:0", small=0):
        self.P = int(n_params)
        self.device = torch.device(device)
        self.ps = tnmps.PauliSum(n, terms)
        self.gates = tnmps.gate_array(circuit)
        self.ctx = []
        for b in sorted({int(batch), int(small)} - {0}):
            m = tnmps.MPSBatch(n, chi, b, dtype=dtype, max_params=self.P, eps=eps,
                               device=self.device)
            th = torch.zeros((b, self.P), dtype=torch.float64, device=self.device)
            e = torch.empty(b, dtype=torch.float64, device=self.device)
            self.ctx.append((b, m, th, e))
        self.batch = int(batch)
        self.evals = 0

    def __call__(self, thetas):
        thetas = np.atleast_2d(np.asarray(thetas, dtype=np.float64))
        out = np.empty(thetas.shape[0])
        for s in range(0, thetas.shape[0], self.batch):
            chunk = thetas[s:s + self.batch]
            k = chunk.shape[0]
            B, m, th, e = next(c for c in self.ctx if c[0] >= k)
            buf = np.empty((B, self.P))
            buf[:k] = chunk
            buf[k:] = chunk[-1]
            th.copy_(torch.from_numpy(buf))
            m.reset()
            m.apply_circuit_dev(self.gates, th)
            m.expect_dev(self.ps, e)
            out[s:s + k] = e[:k].cpu().numpy()
        for c in self.ctx:
            c[1].check()
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
        self.net.check()
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
    best, best_th = np.inf, theta.copy()
    stats = {"iterations": 0, "proposals": 0, "accepted": 0}

    def seen(e, th):
        nonlocal best, best_th
        if e < best:
            best, best_th = e, th.copy()
        hist.append((energy.evals, best))

    while energy.evals < max_evals:
        e0, g, rows, es = param_shift(energy, theta)
        sur.add(rows, es)
        seen(e0, theta)
        if target is not None and best <= target:
            break
        theta, st = opt.propose(theta, g)
        opt.commit(st)
        e = float(energy(theta[None])[0])
        sur.add(theta[None], np.array([e]))
        seen(e, theta)
        for _ in range(sur_steps):
            cand, _ = opt.propose(theta, sur.grad(theta))
            ec = float(energy(cand[None])[0])
            sur.add(cand[None], np.array([ec]))
            stats["proposals"] += 1
            if not ec < e:
                break
            theta, e = cand, ec
            stats["accepted"] += 1
            seen(e, theta)
        stats["iterations"] += 1
        sur.fit(finetune_epochs, finetune_lr, recent=recent, rng=rng)
    return hist, (best, best_th), stats


def evals_to(hist, target):
    for ev, e in hist:
        if e <= target:
            return ev
    return None


def compare(wl, starts=3, budget=200000, lr=0.02, ref_lrs=(0.01, 0.03, 0.05, 0.08),
            ref_budget=300000, n_data=100000, epochs=20, seed=0, dtype="c64", log=None):
    """Surrogate-assisted against plain Adam from several random starts.

    The target of each start is fixed before, and independently of, the two
    compared runs: E* = the lowest energy of long plain-Adam runs from the
    same start at other learning rates (``ref_lrs``, ``ref_budget``
    evaluations each). The compared runs (plain Adam at ``lr``; the surrogate
    method at ``lr`` from the same pretrained surrogate) get the same budget.
    The optimisers evaluate on the ``dtype`` MPS (complex64: its energies are
    within 1e-6 sum|c_k| of the FP64 oracle, far inside the 1e-4 criterion);
    E* and every run's best point are re-evaluated on the complex128 MPS.
    Reported per start: the evaluations each method needs to come within 1e-4
    of E* in the optimisers' form (None: not within the budget) and its best
    energy."""
    P = wl["n_params"]
    args = (wl["n"], wl["chi_max"], wl["eps"], wl["circuit"], P, wl["terms"])
    t0 = time.time()
    rng = np.random.default_rng(4000 + seed)
    gen = MPSEnergy(*args, dtype, 2048)
    X = rng.uniform(-np.pi, np.pi, (n_data, P))
    Y = gen(X)
    t_data = time.time() - t0
    sur = Surrogate(P)
    sur.add(X, Y)
    t1 = time.time()
    train_mse = sur.fit(epochs, 1e-3, restandardise=True)
    t_train = time.time() - t1
    pre = sur.net.get_params().clone()
    mu, sd = sur.mu, sur.sd
    energy = MPSEnergy(*args, dtype, 2 * P + 1, small=1)
    exact = MPSEnergy(*args, "c128", 8)      # complex128 re-evaluation
    rows = []
    for k in range(starts):
        t2 = time.time()
        theta0 = np.random.default_rng(5000 + 100 * seed + k).uniform(-np.pi, np.pi, P)
        refs = []
        for lr_r in ref_lrs:
            energy.evals = 0
            _, b = plain_adam(energy, theta0, lr_r, ref_budget)
            refs.append(b)
        e_star_run = min(b[0] for b in refs)
        best_ref = min(refs, key=lambda b: b[0])
        e_star = float(exact(best_ref[1][None])[0])
        # both compared runs are scored in the optimisers' own form
        target = e_star_run + 1e-4
        energy.evals = 0
        hp, bp = plain_adam(energy, theta0, lr, budget)
        sur.net.set_params(pre)
        sur.mu, sur.sd = mu, sd
        sur.X, sur.Y = X.copy(), Y.copy()
        energy.evals = 0
        hs, bs, st = surrogate_adam(energy, sur, theta0, lr, budget, rng=np.random.default_rng(k))
        row = {"start": k, "E0": float(exact(theta0[None])[0]), "E_star": e_star,
               "E_star_optimiser_form": e_star_run,
               "reference_bests": [float(b[0]) for b in refs],
               "plain_best": float(bp[0]), "surrogate_best": float(bs[0]),
               "plain_best_c128": float(exact(bp[1][None])[0]),
               "surrogate_best_c128": float(exact(np.asarray(bs[1])[None])[0]),
               "plain_evals_to_target": evals_to(hp, target),
               "surrogate_evals_to_target": evals_to(hs, target),
               "plain_evals_to_plain_best": evals_to(hp, bp[0]),
               "surrogate_evals_to_plain_best": evals_to(hs, bp[0]),
               "surrogate_stats": st, "seconds": time.time() - t2}
        rows.append(row)
        if log:
            log(json.dumps(row))
    return {"workload": wl["name"], "params": P, "budget": budget, "lr": lr, "form": dtype,
            "reference": {"learning_rates": list(ref_lrs), "budget": ref_budget},
            "n_data": n_data, "data_s": t_data, "train_s": t_train, "train_mse": train_mse,
            "starts": rows}


def main():
    import argparse
    ap = argparse.ArgumentParser(description="surrogate-assisted vs plain VQE on the MPS")
    ap.add_argument("--workload", default="heis40")
    ap.add_argument("--starts", type=int, default=3)
    ap.add_argument("--n-data", type=int, default=100000)
    ap.add_argument("--budget", type=int, default=200000)
    ap.add_argument("--ref-budget", type=int, default=300000)
    ap.add_argument("--lr", type=float, default=0.02)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--dtype", default="c64", choices=("c64", "c64_bf16split", "c128"))
    a = ap.parse_args()
    wl = inputs.workload(a.workload)
    out = compare(wl, a.starts, a.budget, a.lr, ref_budget=a.ref_budget, n_data=a.n_data,
                  epochs=a.epochs, seed=a.seed, dtype=a.dtype,
                  log=lambda t: print(t, flush=True))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
