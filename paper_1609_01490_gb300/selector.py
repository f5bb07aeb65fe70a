"""Learned map/rho selector: a 2 x 64 MLP cost model trained on the
autotuner's timings with the library's own GPU kernels (tri_mlp_grad,
tri_mlp_adam), queried with tri_mlp_argmin.  Exhaustive autotuning stays the
fallback and the judge of its picks.

Features of a (kernel, n, d, map, rho) candidate (14):
  log2 n, log2 d, log2 rho, log2 of the launched block count under the map,
  kernel one-hot (edm, ca, at), map one-hot (lambda, lambda on P_Delta, BB,
  RB, REC, UTM), log2 of the tile side, standardised with the training set's
  mean and deviation.
Target: log of the measured milliseconds relative to the configuration's
default candidate (lambda, rho = 16): the sizes set a common scale that the
ranking of maps does not depend on, so the model spends its capacity on the
differences between candidates.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np
import torch

from . import tri
from .autotune import KERNELS, MAPS, RHOS, applicable, cand_name

MAP_ORDER = (tri.MAP_LAMBDA, tri.MAP_LAMBDA_PDELTA, tri.MAP_BB, tri.MAP_RB, tri.MAP_REC, tri.MAP_UTM)
DEFAULT = (tri.MAP_LAMBDA, 16)  # the library's default candidate
NFEAT = 14
H1 = H2 = 64


def _tile_side(kernel: str, rho: int, d: int) -> int:
    return {"edm": 4 * rho, "ca": 4 * rho, "at": rho}[kernel]


def _blocks(kernel: str, n: int, d: int, map_id: int, rho: int) -> float:
    m = -(-n // _tile_side(kernel, rho, d))
    if kernel == "at":
        return m ** 3 if map_id == tri.MAP_BB else m * (m + 1) * (m + 2) / 6
    if map_id == tri.MAP_BB:
        return m * m
    if map_id == tri.MAP_RB:
        return m * ((m + 1) // 2 if m % 2 else m // 2 + 1)
    if map_id == tri.MAP_UTM:
        return (n + 1) * n / 2 / (rho * rho)
    return m * (m + 1) / 2


def features(kernel: str, n: int, d: int, map_id: int, rho: int) -> np.ndarray:
    f = np.zeros(NFEAT, dtype=np.float64)
    f[0] = math.log2(n)
    f[1] = math.log2(max(d, 1))
    f[2] = math.log2(rho)
    f[3] = math.log2(max(_blocks(kernel, n, d, map_id, rho), 1.0))
    f[4 + KERNELS.index(kernel)] = 1.0
    f[7 + MAP_ORDER.index(map_id)] = 1.0
    f[13] = math.log2(_tile_side(kernel, rho, d))
    return f


def candidates(kernel: str, n: int, d: int):
    """All applicable (map, rho) of a configuration."""
    return [(m, r) for m in MAPS[kernel] for r in RHOS if applicable(kernel, m, n, r, d)]


def autotune_name(map_id: int, rho: int) -> str:
    return cand_name(map_id, rho)


def parse_name(name: str):
    inv = {v: k for k, v in tri.MAP_NAMES.items()}
    mname, rho = name.split("/")
    return inv[mname], int(rho)


def dataset(table: dict, groups):
    """Rows (features, log(ms / ms of the group's default candidate)) of the
    given groups of a sweep table."""
    X, y = [], []
    for gkey in groups:
        kernel, n, d = gkey.split("|")
        n, d = int(n), int(d)
        tbl = table["groups"][gkey]
        ref = tbl[cand_name(*DEFAULT)]
        for name, ms in tbl.items():
            m, r = parse_name(name)
            X.append(features(kernel, n, d, m, r))
            y.append(math.log(ms / ref))
    return np.array(X), np.array(y)


def split_groups(table: dict, holdout: float = 0.2, seed: int = 1610):
    """Deterministic split of the configurations into training and held-out groups."""
    keys = sorted(table["groups"])
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(keys))
    nh = max(1, int(round(holdout * len(keys))))
    held = sorted(keys[i] for i in perm[:nh])
    train = sorted(keys[i] for i in perm[nh:])
    return train, held


class CostModel:
    """Weights, feature standardisation and the GPU kernels that use them."""

    def __init__(self, theta: np.ndarray, mu: np.ndarray, sd: np.ndarray):
        self.theta = np.asarray(theta, dtype=np.float32)
        self.mu = np.asarray(mu, dtype=np.float64)
        self.sd = np.asarray(sd, dtype=np.float64)
        self._dev = None

    @staticmethod
    def init(seed: int = 0) -> np.ndarray:
        """He-initialised flat parameters (W1, b1, W2, b2, W3, b3)."""
        rng = np.random.default_rng(seed)
        parts = [rng.normal(0, math.sqrt(2.0 / NFEAT), (H1, NFEAT)), np.zeros(H1),
                 rng.normal(0, math.sqrt(2.0 / H1), (H2, H1)), np.zeros(H2),
                 rng.normal(0, math.sqrt(1.0 / H2), (1, H2)), np.zeros(1)]
        return np.concatenate([p.ravel() for p in parts]).astype(np.float32)

    def standardise(self, X: np.ndarray) -> np.ndarray:
        return ((X - self.mu) / self.sd).astype(np.float32)

    def predict(self, X: np.ndarray) -> np.ndarray:
        dev = torch.device("cuda")
        Xd = torch.from_numpy(self.standardise(X)).to(dev)
        th = torch.from_numpy(self.theta).to(dev)
        pred = torch.empty(len(X), device=dev)
        ws = torch.empty(tri.tri_mlp_workspace_size(len(X), H1, H2) // 4 + 1, device=dev)
        tri.tri_mlp_forward(th, Xd, pred, H1, H2, ws)
        return pred.cpu().numpy()

    def pick(self, kernel: str, n: int, d: int):
        """(map, rho) with the smallest predicted time: features,
        standardisation and the argmin all behind the library's tri_select."""
        dev = torch.device("cuda")
        if self._dev is None:
            self._dev = torch.from_numpy(self.theta).to(dev)
        ws = torch.empty(tri.tri_select_workspace_size(H1, H2) // 4 + 64, device=dev)
        return tri.tri_select(self._dev, H1, H2, self.mu, self.sd, KERNELS.index(kernel), n, d, ws)

    def to_json(self) -> dict:
        return {"theta": self.theta.tolist(), "mu": self.mu.tolist(), "sd": self.sd.tolist(), "h1": H1,
                "h2": H2, "nfeat": NFEAT}

    @classmethod
    def from_json(cls, obj: dict) -> "CostModel":
        return cls(np.array(obj["theta"]), np.array(obj["mu"]), np.array(obj["sd"]))


def train(X: np.ndarray, y: np.ndarray, steps: int = 3000, lr: float = 3e-3, seed: int = 0, log=None):
    """Full-batch Adam on the GPU with tri_mlp_grad / tri_mlp_adam.  Returns
    (CostModel, final loss)."""
    mu = X.mean(axis=0)
    sd = X.std(axis=0)
    sd[sd == 0] = 1.0
    model = CostModel(CostModel.init(seed), mu, sd)
    dev = torch.device("cuda")
    Xd = torch.from_numpy(model.standardise(X)).to(dev)
    yd = torch.from_numpy(y.astype(np.float32)).to(dev)
    th = torch.from_numpy(model.theta.copy()).to(dev)
    g = torch.zeros_like(th)
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    loss = torch.zeros(1, device=dev)
    ws = torch.empty(tri.tri_mlp_workspace_size(len(X), H1, H2) // 4 + 1, device=dev)
    for t in range(1, steps + 1):
        tri.tri_mlp_grad(th, Xd, yd, loss, g, H1, H2, ws)
        tri.tri_mlp_adam(th, g, m, v, t, lr)
        if log and (t % 500 == 0 or t == 1):
            log(f"step {t}: loss {float(loss.item()):.5f}")
    torch.cuda.synchronize()
    model.theta = th.cpu().numpy()
    return model, float(loss.item())


def evaluate(model: CostModel, table: dict, groups, default=DEFAULT) -> dict:
    """Mean regret t(pick)/t(best) - 1 over groups for the model, the fixed
    default and the mean random candidate, plus the time a pick takes."""
    reg_model, reg_default, reg_random = [], [], []
    t0 = time.perf_counter()
    picks = {}
    for gkey in groups:
        kernel, n, d = gkey.split("|")
        n, d = int(n), int(d)
        tbl = table["groups"][gkey]
        bestms = min(tbl.values())
        m, r = model.pick(kernel, n, d)
        picks[gkey] = cand_name(m, r)
        reg_model.append(tbl[picks[gkey]] / bestms - 1.0)
        dm = default if kernel != "at" or default[0] in MAPS["at"] else (tri.MAP_LAMBDA, 16)
        reg_default.append(tbl[cand_name(*dm)] / bestms - 1.0)
        reg_random.append(float(np.mean([v / bestms - 1.0 for v in tbl.values()])))
    pick_s = (time.perf_counter() - t0) / max(len(groups), 1)
    tune_ms = float(np.mean([sum(table["groups"][gk].values()) * table.get("reps", 5) for gk in groups]))
    return {"regret_model": float(np.mean(reg_model)), "regret_default": float(np.mean(reg_default)),
            "regret_random": float(np.mean(reg_random)), "picks": picks, "pick_seconds": pick_s,
            "exhaustive_timed_ms_per_group": tune_ms}


def evaluate_loo(table: dict, steps: int = 3000) -> dict:
    """Leave one configuration out: for each group, train on all the others
    and pick for it.  Mean regrets of the model and of the fixed default."""
    keys = sorted(table["groups"])
    reg_model, reg_default, picks = [], [], {}
    for gkey in keys:
        X, y = dataset(table, [k for k in keys if k != gkey])
        model, _ = train(X, y, steps=steps)
        res = evaluate(model, table, [gkey])
        reg_model.append(res["regret_model"])
        reg_default.append(res["regret_default"])
        picks[gkey] = res["picks"][gkey]
    return {"loo_regret_model": float(np.mean(reg_model)), "loo_regret_default": float(np.mean(reg_default)),
            "loo_model_better_or_equal": int(sum(a <= b for a, b in zip(reg_model, reg_default))),
            "loo_groups": len(keys), "loo_picks": picks}


def main(argv=None):
    """python -m paper_1609_01490_gb300.selector sweep OUT.json
       python -m paper_1609_01490_gb300.selector train TABLE.json MODEL.json"""
    import argparse
    from . import autotune
    ap = argparse.ArgumentParser(prog="python -m paper_1609_01490_gb300.selector")
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("sweep", help="time every candidate of the selector sweep")
    a.add_argument("out")
    a.add_argument("--reps", type=int, default=5)
    b = sub.add_parser("train", help="train the cost model on a sweep table, report held-out regret")
    b.add_argument("table")
    b.add_argument("model")
    b.add_argument("--steps", type=int, default=3000)
    args = ap.parse_args(argv)
    if args.cmd == "sweep":
        t0 = time.perf_counter()
        table = autotune.sweep(reps=args.reps, log=print)
        table["seconds"] = time.perf_counter() - t0
        with open(args.out, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        print(f"{sum(len(v) for v in table['groups'].values())} timed candidates in {table['seconds']:.0f} s")
    else:
        with open(args.table) as f:
            table = json.load(f)
        train_g, held = split_groups(table)
        X, y = dataset(table, train_g)
        model, loss = train(X, y, steps=args.steps, log=print)
        res = evaluate(model, table, held)
        res["train_loss"] = loss
        res["train_rows"] = int(len(X))
        res.update(evaluate_loo(table, steps=args.steps))
        with open(args.model, "w") as f:
            json.dump({"model": model.to_json(), "eval": res}, f, indent=1)
        print(json.dumps({k: v for k, v in res.items() if not k.endswith("picks")}, indent=1))


if __name__ == "__main__":
    main()
