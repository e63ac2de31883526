"""Variant tuner of the stage kernels: the paper's evolutionary search (arXiv:1204.4779, section 3)
and a learned cost model that ranks candidates before they are benchmarked.

Variant space (the genome).  The C ABI's hydro_variant_t: tile shape, march length (cells each
thread updates per stage: the threads-per-cell axis), fusion split (dt reduction in RK stage 2's
epilogue, or a separate CFL pass), staging depth (next plane's loads issued one plane ahead, or
at use) and register budget.  In 3D every tile marches along z; in 2D the row tiles (tile_y = 1)
march along y and the one-plane tiles have no march, staging or budget genes (their genomes are
kept canonical so that each variant has one genome).  Every variant computes the same step;
only speed differs.

Score.  As in the paper, an individual is benchmarked several times and scored by the mean and
spread of its cell-updates per second (cups); an individual whose run fails or leaves a
non-finite state scores 0 (the paper's sanity test).

Evolutionary search (section 3.3-3.5).  Births are mutation (one parent, one gene redrawn),
crossover (two parents, two-point) and triangulation (three parents sorted by score into base
< secondary < primary; each gene takes primary's value if it differs from base, else
secondary's, the paper's Table tableTriang), each with probability 1/3.  Parents are drawn with
temperature T, log T uniform on [log sigma_top, log mu_top], with probability proportional to
exp(-max(0, mu_top - mu(I) - sigma_top - sigma(I)) / (T + sigma_top + sigma(I))); a child that is
already in the database is discarded and the draw retried with T multiplied by 1.2.

Learned cost model.  A 3-layer MLP (width 64, FP32) trained by the library's own CUDA kernels
on the tuner's records (variant, grid) -> log time per cell-update; the model-guided search
benchmarks candidates in the order of predicted time, retrains as records arrive, and falls
back to evolutionary births when the model has too few records.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import time
from dataclasses import dataclass, field

import numpy as np

# ------------------------------------------------------------------ the variant space ----

TILES = {
    3: [(32, 8), (32, 4), (64, 4), (16, 16), (32, 16), (16, 8)],
    2: [(32, 8), (64, 4), (16, 16), (32, 16), (64, 1), (128, 1), (256, 1)],
    1: [(128, 1), (256, 1)],
}
MARCHES = [4, 8, 16, 32, 64, 128, 256]
SPLITS = [2, 1]   # hydro_variant_t.split: 2 = fused dt reduction, 1 = separate CFL pass
STAGINGS = [1, 2]
OCCUPANCIES = [2, 3]
MANIFESTS = [1, 2, 3]  # hydro_variant_t.manifest: 1 nothing stored, 2 V stored, 3 fluxes stored
MANIFEST_TILES = [(16, 8), (32, 8), (16, 16)]  # 3D FP32 tiles compiled in the manifest forms


def marching(dim: int, tile) -> bool:
    """Tiles that march: every 3D tile, and the 2D row tiles."""
    return dim == 3 or (dim == 2 and tile[1] == 1)


@dataclass(frozen=True)
class Space:
    """Genes of the variant space of one grid dimension."""
    dim: int

    @property
    def genes(self):
        g = [("tile", TILES[self.dim]), ("march", MARCHES), ("split", SPLITS),
             ("staging", STAGINGS), ("occupancy", OCCUPANCIES)]
        if self.dim == 3:
            return g + [("manifest", MANIFESTS)]
        if self.dim == 2:
            return g
        return [("tile", TILES[self.dim]), ("split", SPLITS)]

    @property
    def sizes(self):
        return [len(v) for _, v in self.genes]

    def canonical(self, genome):
        """The genome with the genes its tile does not use set to their first values; in 3D a
        manifest form only on the tiles compiled with it, with look-ahead staging and the
        three-CTA budget (else nothing stored)."""
        if self.dim == 2 and not marching(2, TILES[2][genome[0]]):
            return (genome[0], 0, genome[2], 0, 0)
        if self.dim == 3 and MANIFESTS[genome[5]] != 1:
            if TILES[3][genome[0]] not in MANIFEST_TILES:
                return tuple(genome[:5]) + (0,)
            return (genome[0], genome[1], genome[2], STAGINGS.index(1), OCCUPANCIES.index(3),
                    genome[5])
        return tuple(genome)

    def all_genomes(self):
        seen, out = set(), []
        for g in itertools.product(*[range(n) for n in self.sizes]):
            c = self.canonical(g)
            if c not in seen:
                seen.add(c)
                out.append(c)
        return out

    def variant(self, genome) -> dict:
        v = {name: vals[g] for (name, vals), g in zip(self.genes, genome)}
        if self.dim == 2 and not marching(2, v["tile"]):
            v = {"tile": v["tile"], "split": v["split"]}
        return v

    def default_genome(self):
        if self.dim == 3:
            d = {"tile": (16, 8), "march": 64, "split": 2, "staging": 1, "occupancy": 3,
                 "manifest": 1}
        elif self.dim == 2:
            d = {"tile": (256, 1), "march": 16, "split": 2, "staging": 1, "occupancy": 3}
        else:
            d = {"tile": (128, 1), "split": 1}
        return tuple(vals.index(d[name]) for name, vals in self.genes)

    def random_genome(self, rng):
        return self.canonical(tuple(int(rng.integers(n)) for n in self.sizes))


def features(space: Space, genome, shape) -> np.ndarray:
    """Input vector of the cost model: one-hot tile, one-hot march (marching tiles), split,
    staging and budget bits, the grid dimension and the log2 sizes of the grid."""
    v = space.variant(genome)
    f = []
    for d in (1, 2, 3):
        tiles = TILES[d]
        f += [1.0 if (space.dim == d and v["tile"] == t) else 0.0 for t in tiles]
    f += [1.0 if v.get("march") == m else 0.0 for m in MARCHES]
    f.append(1.0 if v.get("split", 2) == 1 else 0.0)
    f.append(1.0 if v.get("staging", 1) == 2 else 0.0)
    f.append(1.0 if v.get("occupancy", 2) == 3 else 0.0)
    f += [1.0 if v.get("manifest", 1) == m else 0.0 for m in MANIFESTS[1:]]
    f += [1.0 if space.dim == d else 0.0 for d in (1, 2, 3)]
    n = list(shape) + [1] * (3 - len(shape))
    f += [math.log2(max(x, 1)) / 10.0 for x in n]
    f.append(math.log2(max(1, int(np.prod(shape)))) / 30.0)
    f.append(min(1.0, n[2] / 512.0) if space.dim == 3 else 0.0)
    return np.array(f, dtype=np.float64)


N_FEATURES = len(features(Space(3), Space(3).default_genome(), (8, 8, 8)))

# --------------------------------------------------------------------- records ----------


@dataclass
class Record:
    dim: int
    shape: tuple
    genome: tuple
    mu: float        # mean cups
    sigma: float     # spread of cups over the repetitions
    ok: bool = True
    seconds: float = 0.0  # wall-clock the benchmark took

    def to_json(self) -> str:
        return json.dumps({"dim": self.dim, "shape": list(self.shape), "genome": list(self.genome),
                           "mu": self.mu, "sigma": self.sigma, "ok": self.ok,
                           "seconds": self.seconds})

    @staticmethod
    def from_json(s: str) -> "Record":
        d = json.loads(s)
        genome = tuple(d["genome"])
        if d["dim"] == 3 and len(genome) == 5:  # records from before the manifest gene
            genome = genome + (0,)
        return Record(d["dim"], tuple(d["shape"]), genome, d["mu"], d["sigma"],
                      d.get("ok", True), d.get("seconds", 0.0))


class DB:
    """Append-only record store (JSON lines), resumable like the paper's database."""

    def __init__(self, path: str | None = None):
        self.path = path
        self.records: list[Record] = []
        if path and os.path.exists(path):
            with open(path) as f:
                self.records = [Record.from_json(l) for l in f if l.strip()]

    def add(self, r: Record):
        self.records.append(r)
        if self.path:
            with open(self.path, "a") as f:
                f.write(r.to_json() + "\n")

    def for_grid(self, shape):
        return [r for r in self.records if tuple(r.shape) == tuple(shape)]


# --------------------------------------------------------------- benchmarking -----------


class Benchmark:
    """Times a variant on one grid: `reps` repetitions of `steps` RK steps each (CUDA events),
    after one warm-up step; the initial state is restored before every repetition.  Returns a
    Record with the mean and spread of cups; a failed or non-finite run scores 0."""

    def __init__(self, shape, dtype="f32", reps: int = 5, steps: int = 2, seed: int = 1204477905):
        import torch

        from . import hydro, inputs
        self.torch, self.hydro = torch, hydro
        self.shape = tuple(int(s) for s in shape)
        self.dim = len(self.shape)
        self.space = Space(self.dim)
        self.reps, self.steps = reps, steps
        self.dt = torch.float32 if dtype == "f32" else torch.float64
        if self.dim == 3:
            nx, ny, nz = self.shape
            if nx == ny == nz:
                V = inputs.blast_3d_torch(nx, 8.0, device="cuda")
            else:
                V = torch.from_numpy(inputs.blast_3d(shape=self.shape, radius_cells=8.0)).cuda()
            self.gamma = 1.4
        elif self.dim == 2:
            V = torch.from_numpy(inputs.kh_2d(self.shape[0], seed=seed, ny=self.shape[1])).cuda()
            self.gamma = 5.0 / 3.0
        else:
            V = torch.from_numpy(inputs.sod_1d(self.shape[0])).cuda()
            self.gamma = 1.4
        self.U0 = hydro.prim_to_cons(V, self.gamma).to(self.dt).contiguous()
        del V
        self.U = torch.empty_like(self.U0)
        self.ncell = int(np.prod(self.shape))

    def __call__(self, genome) -> Record:
        torch, hydro = self.torch, self.hydro
        v = self.space.variant(genome)
        t_start = time.perf_counter()
        cups = []
        ok = True
        try:
            S = hydro.Solver(self.shape, self.gamma, bc="periodic", dtype=self.dt, cfl=0.4,
                             variant=dict(tile=v["tile"], march=v.get("march", 0),
                                          split=v.get("split", 0), staging=v.get("staging", 0),
                                          occupancy=v.get("occupancy", 0),
                                          manifest=v.get("manifest", 0)))
            self.U.copy_(self.U0)
            S.step(self.U, 1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for _ in range(self.reps):
                self.U.copy_(self.U0)
                torch.cuda.synchronize()
                e0.record()
                _, done = S.step(self.U, self.steps)
                e1.record()
                torch.cuda.synchronize()
                if done != self.steps:
                    raise RuntimeError("steps missing")
                cups.append(self.ncell * self.steps / (e0.elapsed_time(e1) * 1e-3))
            ok = bool(torch.isfinite(self.U).all().item()) and not torch.equal(self.U, self.U0)
            S.close()
        except Exception:
            ok = False
        if not ok or not cups:
            return Record(self.dim, self.shape, tuple(genome), 0.0, 0.0, False,
                          time.perf_counter() - t_start)
        return Record(self.dim, self.shape, tuple(genome), float(np.mean(cups)),
                      float(np.std(cups)), True, time.perf_counter() - t_start)


# ------------------------------------------------------------ evolutionary search --------


def triangulate(base, secondary, primary):
    """Child of three parents (ascending score): adopt primary's change from base if any,
    else secondary's (the paper's Table tableTriang, gene by gene)."""
    return tuple(p if p != b else s for b, s, p in zip(base, secondary, primary))


class Evolution:
    """The paper's search over one grid's variant space; `evaluate(genome) -> Record`."""

    def __init__(self, space: Space, rng, records=None):
        self.space = space
        self.rng = rng
        self.scores: dict[tuple, tuple[float, float]] = {}
        for r in records or []:
            self.scores[tuple(r.genome)] = (r.mu if r.ok else 0.0, r.sigma if r.ok else 0.0)

    def top(self):
        g = max(self.scores, key=lambda k: self.scores[k][0])
        return g, self.scores[g]

    def draw(self, T: float, exclude=()):
        _, (mu_t, sig_t) = self.top()
        keys = [k for k in self.scores if k not in exclude]
        if not keys:
            return None
        # exponents of the draw probabilities; the largest is subtracted before exponentiating
        # (the same distribution, without every weight underflowing when the spreads are tiny)
        x = np.array([-max(0.0, mu_t - self.scores[k][0] - sig_t - self.scores[k][1]) /
                      max(T + sig_t + self.scores[k][1], 1e-30) for k in keys])
        w = np.exp(x - x.max())
        w = w / w.sum()
        return keys[int(self.rng.choice(len(keys), p=w))]

    def temperature(self) -> float:
        _, (mu_t, sig_t) = self.top()
        lo = math.log(max(sig_t, 1e-6 * max(mu_t, 1e-30), 1e-30))
        hi = math.log(max(mu_t, 1e-30))
        if hi <= lo:
            return math.exp(hi)
        return math.exp(self.rng.uniform(lo, hi))

    def birth(self, max_retries: int = 200):
        """A genome not yet in the database (or None when the space is exhausted)."""
        sizes = self.space.sizes
        if len(self.scores) >= len(self.space.all_genomes()):
            return None
        T = self.temperature()
        for _ in range(max_retries):
            kind = self.rng.integers(3)
            child = None
            if kind == 0 or len(self.scores) < 2:
                a = self.draw(T)
                gi = int(self.rng.integers(len(sizes)))
                choices = [x for x in range(sizes[gi]) if x != a[gi]]
                if choices:
                    child = list(a)
                    child[gi] = int(self.rng.choice(choices))
                    child = tuple(child)
            elif kind == 1 or len(self.scores) < 3:
                a = self.draw(T)
                b = self.draw(T, exclude=(a,))
                i, j = sorted(self.rng.choice(len(sizes) + 1, 2, replace=False))
                child = tuple(b[k] if i <= k < j else a[k] for k in range(len(sizes)))
            else:
                a = self.draw(T)
                b = self.draw(T, exclude=(a,))
                c = self.draw(T, exclude=(a, b))
                base, sec, prim = sorted((a, b, c), key=lambda k: self.scores[k][0])
                child = triangulate(base, sec, prim)
            if child is not None:
                child = self.space.canonical(child)
                if child not in self.scores:
                    return child
            T *= 1.2
        # exhausted retries: any unseen genome
        unseen = [g for g in self.space.all_genomes() if g not in self.scores]
        return unseen[int(self.rng.integers(len(unseen)))] if unseen else None

    def add(self, r: Record):
        self.scores[tuple(r.genome)] = (r.mu if r.ok else 0.0, r.sigma if r.ok else 0.0)


def _over_budget(done, spent, budget_evals, budget_seconds) -> bool:
    """True if another benchmark would exceed the budget (its cost estimated as the mean of
    the benchmarks so far)."""
    if budget_evals is not None and len(done) >= budget_evals:
        return True
    if budget_seconds is not None:
        est = np.mean([r.seconds for r in done]) if done else 0.0
        if spent + est > budget_seconds:
            return True
    return False


def time_to_best(done, t_marks):
    """Wall-clock at which the final best record was first reached (None if nothing was
    benchmarked)."""
    if not t_marks:
        return None
    best = max(r.mu for r in done)
    for r, t in zip(done, t_marks):
        if r.mu >= best:
            return t
    return t_marks[-1]


def evolve(space, evaluate, rng, budget_evals=None, budget_seconds=None, initial=None, db=None,
           marks=None, clock=time.perf_counter):
    """Plain evolutionary search; returns (best Record, list of Records, seconds spent).
    `marks`, if a list, receives the wall-clock after each benchmark; `clock` reads it."""
    ev = Evolution(space, rng)
    done, t0 = [], clock()
    queue = list(initial or [space.default_genome()])
    while True:
        spent = clock() - t0
        if _over_budget(done, spent, budget_evals, budget_seconds):
            break
        g = queue.pop(0) if queue else ev.birth()
        if g is None:
            break
        if g in ev.scores:
            continue
        r = evaluate(g)
        ev.add(r)
        done.append(r)
        if marks is not None:
            marks.append(clock() - t0)
        if db is not None:
            db.add(r)
    best = max(done, key=lambda r: r.mu)
    return best, done, clock() - t0


# ------------------------------------------------------------ learned cost model ----------


def training_set(records, exclude_shape=None):
    X, y = [], []
    for r in records:
        if not r.ok or r.mu <= 0 or (exclude_shape is not None and tuple(r.shape) == tuple(exclude_shape)):
            continue
        X.append(features(Space(r.dim), r.genome, r.shape))
        y.append(-math.log(r.mu))  # log seconds per cell-update
    return np.array(X), np.array(y)


class CostModel:
    """Standardised-target wrapper of an MLP with predict(X) and train(X, t, epochs, lr)."""

    def __init__(self, make_mlp, epochs: int = 800, lr: float = 3e-3):
        self.make_mlp, self.epochs, self.lr = make_mlp, epochs, lr
        self.net = None
        self.mean, self.std = 0.0, 1.0

    def fit(self, X, y, epochs=None, warm: bool = False):
        self.mean, self.std = float(np.mean(y)), float(np.std(y) or 1.0)
        if self.net is None or not warm:
            self.net = self.make_mlp(X.shape[1])
        return self.net.train(X, (y - self.mean) / self.std, epochs or self.epochs, self.lr)

    def predict(self, X):
        return self.net.predict(X) * self.std + self.mean


def spearman(a, b) -> float:
    ra = np.argsort(np.argsort(a))
    rb = np.argsort(np.argsort(b))
    if len(a) < 2:
        return float("nan")
    return float(np.corrcoef(ra, rb)[0, 1])


def model_guided(space, shape, evaluate, model: CostModel, records, rng, budget_evals=None,
                 budget_seconds=None, retrain_every: int = 4, min_records: int = 20, db=None,
                 pretrained: bool = False, marks=None, clock=time.perf_counter):
    """Benchmark candidates in the order of the model's predicted time, retraining on the
    records as they arrive; evolutionary births when the model has too few records.
    `pretrained`: the model was already fitted on `records` (offline, before the target was
    known); otherwise the first fit counts against the budget.
    Returns (best Record, list of Records, seconds spent including any training)."""
    t0 = clock()
    pool = list(records)
    ev = Evolution(space, rng)
    done = []
    cands = space.all_genomes()
    Xc = np.array([features(space, g, shape) for g in cands])
    trained = pretrained
    per_epoch = None  # measured seconds per training epoch
    while True:
        spent = clock() - t0
        if _over_budget(done, spent, budget_evals, budget_seconds):
            break
        retrain = trained and len(done) > 0 and len(done) % retrain_every == 0
        if retrain and budget_seconds is not None and per_epoch is not None:
            # skip a retraining that would leave no time for the next benchmark
            epochs = max(100, model.epochs // 4)
            if spent + per_epoch * epochs + np.mean([r.seconds for r in done]) > budget_seconds:
                retrain = False
        if not trained or retrain:
            X, y = training_set(pool)
            if len(y) >= min_records:
                epochs = model.epochs if not trained else max(100, model.epochs // 4)
                t1 = clock()
                model.fit(X, y, epochs=epochs, warm=trained)
                per_epoch = (clock() - t1) / epochs
                trained = True
            if _over_budget(done, clock() - t0, budget_evals, budget_seconds):
                break
        if trained:
            pred = model.predict(Xc)
            order = np.argsort(pred)
            g = next((cands[i] for i in order if cands[i] not in ev.scores), None)
        else:
            g = space.default_genome() if not done else ev.birth()
        if g is None:
            break
        r = evaluate(g)
        ev.add(r)
        done.append(r)
        pool.append(r)
        if marks is not None:
            marks.append(clock() - t0)
        if db is not None:
            db.add(r)
    if not done:  # the budget ran out during the first training: nothing benchmarked
        best = Record(space.dim, tuple(shape), tuple(space.default_genome()), 0.0, 0.0, False, 0.0)
        return best, [best], clock() - t0
    best = max(done, key=lambda r: r.mu)
    return best, done, clock() - t0


def gpu_mlp_factory(hidden: int = 64, seed: int = 0):
    from .costmodel import MLP
    return lambda d: MLP(d, hidden, seed=seed)


# --------------------------------------------------------------------- driver -----------

TRAIN_SHAPES = ([(n, n, n) for n in (32, 48, 64, 80, 96, 160, 192, 224, 256, 320, 384)] +
                [(256, 128, 64), (128, 256, 96), (384, 192, 128)] +
                [(n, n) for n in (256, 512, 768, 1024, 1536, 3072, 4096)])
TARGETS = [(512, 512, 512), (2048, 2048), (128, 128, 128)]


def collect(db: DB, shapes, per_shape: int, rng, reps: int = 5, steps: int = 2, log=print):
    """Tuner measurements on training grids: `per_shape` random distinct variants each (all of
    them when the space is smaller)."""
    for sh in shapes:
        bench = Benchmark(sh, reps=reps, steps=steps)
        genomes = bench.space.all_genomes()
        have = {r.genome for r in db.for_grid(sh)}
        order = [genomes[i] for i in rng.permutation(len(genomes))]
        todo = [g for g in order if g not in have][:max(0, per_shape - len(have))]
        for g in todo:
            db.add(bench(g))
        log(f"collected {len(todo)} records on {sh} (total {len(db.records)})")
        del bench


def compare(db: DB, target, ga_evals: int, rng_seed: int, reps: int = 10, steps: int = 2,
            hidden: int = 64):
    """Plain evolutionary search vs the model-guided search on `target`.

    The plain search gets `ga_evals` benchmarks (wall-clock W).  The cost model is trained
    offline on the other grids' records only (its training time is reported separately: it
    happens before the target is known and serves every target); the model-guided search then
    gets 0.25 W (and, separately, W), its incremental retraining counted in its budget.  Also
    reported: the plain search with 0.25 W, each search's time to its best, and the model's
    ranking error on everything the plain search measured (Spearman, top-1 regret)."""
    bench = Benchmark(target, reps=reps, steps=steps)
    space = bench.space
    others = [r for r in db.records if tuple(r.shape) != tuple(target)]
    X, y = training_set(others)
    t_train0 = time.perf_counter()
    base = CostModel(gpu_mlp_factory(hidden, seed=rng_seed))
    losses = base.fit(X, y)
    train_s = time.perf_counter() - t_train0
    marks = []
    # the plain searches start from a seeded random variant: the library defaults came out of
    # earlier tuning, and starting there would hand them the answer
    start = [space.random_genome(np.random.default_rng(rng_seed + 7))]
    ga_best, ga_done, ga_s = evolve(space, bench, np.random.default_rng(rng_seed),
                                    budget_evals=ga_evals, marks=marks, initial=start)
    ok = [r for r in ga_done if r.ok]
    pred = base.predict(np.array([features(space, r.genome, target) for r in ok]))
    meas = np.array([-math.log(r.mu) for r in ok])
    out = {"target": list(target), "records_used": int(len(y)), "offline_train_seconds": train_s,
           "train_loss_first_last": [float(losses[0]), float(losses[-1])],
           "ga": {"evals": len(ga_done), "seconds": ga_s, "time_to_best": time_to_best(ga_done, marks),
                  "best_cups": ga_best.mu, "best_sigma": ga_best.sigma,
                  "best_variant": space.variant(ga_best.genome)},
           "spearman_pred_vs_measured_on_ga_set": spearman(pred, meas),
           "top1_regret_on_ga_set": float(ga_best.mu / ok[int(np.argmin(pred))].mu - 1.0)}
    for frac in (0.25, 1.0):
        cm = CostModel(gpu_mlp_factory(hidden, seed=rng_seed))
        cm.net, cm.mean, cm.std = base.net, base.mean, base.std  # the offline-trained model
        mk = []
        b, done, s = model_guided(space, target, bench, cm, others, np.random.default_rng(rng_seed),
                                  budget_seconds=frac * ga_s, pretrained=True, marks=mk)
        out[f"model_{int(frac * 100)}pct"] = {
            "evals": len(done), "seconds": s, "time_to_best": time_to_best(done, mk),
            "best_cups": b.mu, "best_sigma": b.sigma, "best_variant": space.variant(b.genome),
            "matches_or_beats_ga": bool(b.mu >= ga_best.mu - (ga_best.sigma + b.sigma))}
        base = CostModel(gpu_mlp_factory(hidden, seed=rng_seed))  # fresh copy for the next run
        base.fit(X, y)
    mk = []
    nb, ndone, ns = evolve(space, bench, np.random.default_rng(rng_seed + 1),
                           budget_seconds=0.25 * ga_s, marks=mk, initial=start)
    out["plain_25pct"] = {"evals": len(ndone), "seconds": ns, "time_to_best": time_to_best(ndone, mk),
                          "best_cups": nb.mu, "best_variant": space.variant(nb.genome),
                          "matches_ga": bool(nb.mu >= ga_best.mu - (ga_best.sigma + nb.sigma))}
    for r in ga_done:
        db.add(r)
    return out


def study(db: DB, target, seeds: int, ga_evals: int, reps: int = 10, steps: int = 2,
          hidden: int = 64, frac: float = 0.25, log=print, bench=None, mlp_factory=None,
          clock=time.perf_counter):
    """Several seeds of three searches on `target`:

      plain_W      the plain evolutionary search with `ga_evals` benchmarks; its wall-clock
                   is that seed's W;
      plain_frac   the plain search with frac * W of wall-clock;
      model_frac   the model-guided search with frac * W of wall-clock, its clock INCLUDING
                   training the cost model from scratch (on the other grids' records, before
                   its first benchmark) and every retraining.

    Every search starts from the same seeded random variant.  A seed's model search 'matches'
    when its best is within sigma_W + sigma of the plain_W best.  Returns per-seed records and,
    per arm, the mean and standard deviation of the best rate and of the time to best.
    `bench` (an evaluator with a .space), `mlp_factory(seed)` and `clock` replace the GPU
    benchmark, the GPU MLP and the wall-clock (tests)."""
    bench = bench if bench is not None else Benchmark(target, reps=reps, steps=steps)
    mlp_factory = mlp_factory or (lambda seed: gpu_mlp_factory(hidden, seed=seed))
    space = bench.space
    others = [r for r in db.records if tuple(r.shape) != tuple(target)]
    runs = []
    for s in range(seeds):
        start = [space.random_genome(np.random.default_rng(1000 + s))]
        mk = []
        ga_best, ga_done, W = evolve(space, bench, np.random.default_rng(s), budget_evals=ga_evals,
                                     marks=mk, initial=start, clock=clock)
        rec = {"seed": s, "W": W,
               "plain_W": {"evals": len(ga_done), "seconds": W, "best": ga_best.mu,
                           "sigma": ga_best.sigma, "time_to_best": time_to_best(ga_done, mk),
                           "variant": space.variant(ga_best.genome)}}
        mk = []
        nb, nd, ns = evolve(space, bench, np.random.default_rng(10_000 + s),
                            budget_seconds=frac * W, marks=mk, initial=start, clock=clock)
        rec["plain_frac"] = {"evals": len(nd), "seconds": ns, "best": nb.mu, "sigma": nb.sigma,
                             "time_to_best": time_to_best(nd, mk),
                             "variant": space.variant(nb.genome)}
        mk = []
        cm = CostModel(mlp_factory(s))
        mb, md, ms = model_guided(space, target, bench, cm, others, np.random.default_rng(s),
                                  budget_seconds=frac * W, pretrained=False, marks=mk,
                                  clock=clock)
        rec["model_frac"] = {"evals": len(mk), "seconds": ms, "best": mb.mu, "sigma": mb.sigma,
                             "time_to_best": time_to_best(md, mk),
                             "variant": space.variant(mb.genome),
                             "matches_plain_W": bool(mb.mu >= ga_best.mu - (ga_best.sigma + mb.sigma))}
        runs.append(rec)
        log(f"{target} seed {s}: W {W:.2f} s  plain_W {ga_best.mu / 1e9:.3f} G  "
            f"plain_frac {nb.mu / 1e9:.3f} G  model_frac {mb.mu / 1e9:.3f} G "
            f"({len(mk)} benchmarks, {ms:.2f} s)")
    summary = {}
    for arm in ("plain_W", "plain_frac", "model_frac"):
        b = np.array([r[arm]["best"] for r in runs])
        t = np.array([r[arm]["time_to_best"] if r[arm]["time_to_best"] is not None else np.nan
                      for r in runs])
        summary[arm] = {"best_mean": float(b.mean()), "best_sd": float(b.std(ddof=1)) if len(b) > 1 else 0.0,
                        "ttb_mean": float(np.nanmean(t)) if np.isfinite(t).any() else None,
                        "ttb_sd": float(np.nanstd(t, ddof=1)) if np.isfinite(t).sum() > 1 else 0.0}
    summary["model_matches"] = int(sum(r["model_frac"]["matches_plain_W"] for r in runs))
    summary["seeds"] = len(runs)
    summary["W_mean"] = float(np.mean([r["W"] for r in runs]))
    return {"target": list(target), "frac": frac, "ga_evals": ga_evals, "reps": reps,
            "steps": steps, "records_used": len(others), "summary": summary, "runs": runs}


BATCH_VARIANTS = ([((32, 8), 0), ((16, 16), 0)] +
                  [(t, m) for t in ((32, 1), (64, 1), (128, 1)) for m in (8, 16, 32, 64)])


def sweep_batched(reps: int = 3, steps: int = 10, seed: int = 1204477904):
    """Cell-updates/s of the batched configuration (4096 grids, sides log-uniform on [32, 512],
    seeded smooth data, FP32) for each (tile, march) of BATCH_VARIANTS: best of `reps` runs of
    `steps` graph-replayed steps, CUDA events around each run."""
    import torch

    from . import hydro, inputs
    shapes = [tuple(int(v) for v in s) for s in inputs.batch_shapes()]
    P = np.concatenate([inputs.batch_grid(nx, ny, seed, i).reshape(4, -1)
                        for i, (nx, ny) in enumerate(shapes)], 1)
    U64 = hydro.prim_to_cons(torch.from_numpy(P).cuda().view(4, 1, -1), 1.4).view(4, -1)
    out = []
    for tile, march in BATCH_VARIANTS:
        B = hydro.BatchSolver(shapes, 1.4, dtype=torch.float32, tile=tile, march=march)
        U = U64.float().contiguous()
        B.step(U, steps)  # capture the graphs
        best = None
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            B.step(U, steps, sync=False)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out.append({"tile": list(tile), "march": march,
                    "cups": U.shape[1] * steps / (best * 1e-3)})
        B.close()
    return sorted(out, key=lambda r: -r["cups"])


def sweep(shape, reps: int = 5, steps: int = 20):
    """Every variant of the grid's space (Benchmark: `reps` runs of `steps` steps from the same
    initial state), sorted by mean cell-updates/s."""
    bench = Benchmark(shape, reps=reps, steps=steps)
    recs = [bench(g) for g in bench.space.all_genomes()]
    return sorted(({"variant": bench.space.variant(r.genome), "cups": r.mu, "sigma": r.sigma,
                    "ok": r.ok} for r in recs), key=lambda d: -d["cups"])


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("command", choices=("collect", "compare", "study", "sweep"))
    ap.add_argument("--db", default=None)
    ap.add_argument("--shape", type=int, nargs="+", default=None,
                    help="sweep: the grid (nx [ny [nz]]); omitted: the batched configuration")
    ap.add_argument("--per-shape", type=int, default=150)
    ap.add_argument("--ga-evals", type=int, default=60)
    ap.add_argument("--seed", type=int, default=1204477905)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--out", default=None)
    ap.add_argument("--seeds", type=int, default=5, help="study: seeds per target")
    a = ap.parse_args(argv)
    if a.command == "sweep":
        res = sweep(tuple(a.shape), a.reps, a.steps) if a.shape else sweep_batched(a.reps, a.steps)
        text = json.dumps({"shape": a.shape or "batched 4096 grids", "results": res}, indent=1)
        print(text)
        if a.out:
            with open(a.out, "w") as f:
                f.write(text + "\n")
        return
    if not a.db:
        ap.error("--db is required for collect and compare")
    db = DB(a.db)
    if a.command == "collect":
        collect(db, TRAIN_SHAPES, a.per_shape, np.random.default_rng(a.seed), a.reps, a.steps)
        return
    if a.command == "study":
        results = [study(db, t, a.seeds, a.ga_evals, a.reps, a.steps) for t in TARGETS]
        text = json.dumps({"records_in_db": len(db.records), "results": results}, indent=1)
        print(text)
        if a.out:
            with open(a.out, "w") as f:
                f.write(text + "\n")
        return
    results = [compare(db, t, a.ga_evals, a.seed, a.reps, a.steps) for t in TARGETS]
    text = json.dumps({"records_in_db": len(db.records), "results": results}, indent=1)
    print(text)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text + "\n")


if __name__ == "__main__":
    main()
