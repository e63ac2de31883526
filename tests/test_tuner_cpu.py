"""Host logic of the variant tuner: the paper's triangulation table, the temperature draw,
births that avoid the database, the evolutionary search and the model-guided search on a
synthetic cost landscape (the MLP here is the FP64 CPU oracle of the cost model)."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_1204_4779_gb300 import tuner as T


def test_triangulation_truth_table():
    """Table tableTriang of the paper: (base, secondary, primary) -> child, bit by bit."""
    table = {(0, 0, 0): 0, (0, 0, 1): 1, (0, 1, 0): 1, (0, 1, 1): 1,
             (1, 0, 0): 0, (1, 0, 1): 0, (1, 1, 0): 0, (1, 1, 1): 1}
    bases, secs, prims = zip(*table.keys())
    child = T.triangulate(bases, secs, prims)
    assert child == tuple(table.values())
    # multi-valued genes: primary's change wins, else secondary's
    assert T.triangulate((2, 5, 1), (3, 5, 1), (2, 6, 1)) == (3, 6, 1)


def test_space_and_features():
    s3 = T.Space(3)
    # 3D: every tile x march x split x staging x budget storing nothing, plus the two manifest
    # forms on the three tiles compiled with them (look-ahead staging, three-CTA budget)
    assert len(s3.all_genomes()) == 6 * 7 * 2 * 2 * 2 + 3 * 7 * 2 * 2
    assert s3.variant(s3.default_genome()) == {"tile": (16, 8), "march": 64, "split": 2,
                                               "staging": 1, "occupancy": 3, "manifest": 1}
    for g in s3.all_genomes():
        v = s3.variant(g)
        if v["manifest"] != 1:
            assert v["tile"] in T.MANIFEST_TILES and v["staging"] == 1 and v["occupancy"] == 3
    old = T.Record.from_json('{"dim": 3, "shape": [64, 64, 64], "genome": [0, 4, 0, 0, 1], '
                             '"mu": 1.0, "sigma": 0.0}')
    assert old.genome == (0, 4, 0, 0, 1, 0) and s3.variant(old.genome)["manifest"] == 1
    f = T.features(s3, s3.default_genome(), (512, 512, 512))
    assert f.shape == (T.N_FEATURES,)
    f2 = T.features(T.Space(2), T.Space(2).default_genome(), (2048, 2048))
    assert f2.shape == (T.N_FEATURES,) and not np.array_equal(f, f2)
    assert len({tuple(T.features(s3, g, (64, 64, 64))) for g in s3.all_genomes()}) == 336 + 84
    # 2D: four one-plane tiles (tile and split genes only) and three row tiles with every gene
    s2 = T.Space(2)
    g2 = s2.all_genomes()
    assert len(g2) == 4 * 2 + 3 * 7 * 2 * 2 * 2 and len(set(g2)) == len(g2)
    assert s2.variant(s2.default_genome()) == {"tile": (256, 1), "march": 16, "split": 2,
                                               "staging": 1, "occupancy": 3}
    assert all(set(s2.variant(g)) == {"tile", "split"} for g in g2 if s2.variant(g)["tile"][1] > 1)
    assert len({tuple(T.features(s2, g, (64, 64))) for g in g2}) == len(g2)
    rng = np.random.default_rng(3)
    assert all(s2.random_genome(rng) in set(g2) for _ in range(200))


def test_draw_prefers_high_scores_at_low_temperature():
    rng = np.random.default_rng(0)
    ev = T.Evolution(T.Space(2), rng)
    ev.scores = {(0, 0): (100.0, 1.0), (1, 0): (50.0, 1.0), (2, 0): (10.0, 1.0)}
    picks = [ev.draw(1e-3) for _ in range(200)]
    assert picks.count((0, 0)) == 200
    picks = [ev.draw(1e6) for _ in range(3000)]
    assert min(picks.count(k) for k in ev.scores) > 700  # nearly uniform when hot
    # differences inside the noise are ignored
    ev.scores = {(0, 0): (100.0, 5.0), (1, 0): (95.0, 5.0)}
    picks = [ev.draw(1e-3) for _ in range(2000)]
    assert 800 < picks.count((1, 0)) < 1200


def test_births_are_new_and_exhaust_the_space():
    rng = np.random.default_rng(1)
    space = T.Space(2)
    ev = T.Evolution(space, rng)
    seen = set()
    for g in space.all_genomes()[:3]:
        ev.add(T.Record(2, (64, 64), g, float(rng.uniform(1, 2)), 0.01))
        seen.add(g)
    while True:
        g = ev.birth()
        if g is None:
            break
        assert g not in seen
        seen.add(g)
        ev.add(T.Record(2, (64, 64), g, float(rng.uniform(1, 2)), 0.01))
    assert seen == set(space.all_genomes())


def synthetic_cups(space, genome, shape, noise_rng=None):
    """A cost landscape with structure shared across grid sizes: tile, march and the manifest
    form matter most, the split and staging a little; larger grids favour longer marches."""
    v = space.variant(genome)
    tile_cost = {(32, 8): 0.12, (32, 4): 0.15, (64, 4): 0.1, (16, 16): 0.0, (32, 16): 0.2,
                 (16, 8): 0.3}[v["tile"]]
    nz = shape[2]
    best_march = min(256, max(4, nz // 4))
    march_cost = 0.05 * (math.log2(v["march"]) - math.log2(best_march)) ** 2
    manifest_cost = {1: 0.0, 2: 0.15, 3: 0.35}[v.get("manifest", 1)]  # HBM round trips cost
    logt = (-23.0 + tile_cost + march_cost + 0.08 * (v["split"] == 1) + 0.04 * (v["staging"] == 2)
            - 0.03 * (v["occupancy"] == 3) + manifest_cost)
    if noise_rng is not None:
        logt += noise_rng.normal(0, 0.005)
    return math.exp(-logt)


class NumpyMLP:
    def __init__(self, d, hidden=16, seed=0):
        rng = np.random.default_rng(seed)
        self.d, self.h = d, hidden
        self.p = rng.normal(0, 0.3, M.param_count(d, hidden))
        self.m = np.zeros_like(self.p)
        self.v = np.zeros_like(self.p)
        self.k = 0

    def train(self, X, t, epochs, lr):
        for _ in range(epochs):
            self.k += 1
            g = M.gradient(self.p, X, t, self.d, self.h)
            self.p, self.m, self.v = M.adam_step(self.p, g, self.m, self.v, self.k, lr)
        return np.array([M.loss(self.p, X, t, self.d, self.h)])

    def predict(self, X):
        return M.forward(self.p, X, self.d, self.h)[0]


def _evaluator(space, shape, seed):
    rng = np.random.default_rng(seed)

    def ev(g):
        mu = synthetic_cups(space, g, shape, rng)
        return T.Record(space.dim, shape, g, mu, 0.002 * mu, True, 0.1)
    return ev


def test_evolution_finds_the_optimum_of_a_synthetic_landscape():
    space = T.Space(3)
    shape = (256, 256, 256)
    best, done, _ = T.evolve(space, _evaluator(space, shape, 3), np.random.default_rng(3),
                             budget_evals=80)
    truth = max(synthetic_cups(space, g, shape) for g in space.all_genomes())
    assert best.mu >= 0.97 * truth
    assert len({r.genome for r in done}) == len(done)


@pytest.mark.slow
def test_model_guided_search_gains_over_search_without_the_model():
    """Trained on other grid sizes, the model ranks the target's candidates so that a few
    benchmarks find the best variant; without the model (the plain search) the same few
    benchmarks do worse on average."""
    space = T.Space(3)
    train_shapes = [(n, n, n) for n in (32, 48, 64, 96, 160, 256)]
    records = []
    rng = np.random.default_rng(7)
    for sh in train_shapes:
        ev = _evaluator(space, sh, 11)
        for g in rng.permutation(len(space.all_genomes()))[:80]:
            records.append(ev(space.all_genomes()[g]))
    target = (512, 512, 512)
    truth = max(synthetic_cups(space, g, target) for g in space.all_genomes())
    budget = 8
    model_best, plain_best = [], []
    for seed in range(3):
        cm = T.CostModel(lambda d: NumpyMLP(d, 16, seed), epochs=400, lr=1e-2)
        b, _, _ = T.model_guided(space, target, _evaluator(space, target, seed), cm, records,
                                 np.random.default_rng(seed), budget_evals=budget,
                                 retrain_every=100)
        model_best.append(b.mu / truth)
        b2, _, _ = T.evolve(space, _evaluator(space, target, seed), np.random.default_rng(seed),
                            budget_evals=budget)
        plain_best.append(b2.mu / truth)
    assert min(model_best) >= 0.97
    assert np.mean(model_best) > np.mean(plain_best)


class _VirtualClock:
    """Simulated wall-clock: each benchmark costs 0.1 s and the model's training 0.3 s per 800
    epochs."""

    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


def test_study_arms_budgets_and_summary():
    """The multi-seed study on a synthetic landscape with a simulated clock: per seed the plain
    search's W, the plain and model-guided searches within a quarter of it (the model's training
    counted in its clock), and the per-arm means."""
    space = T.Space(3)
    clock = _VirtualClock()
    db = T.DB(None)
    rng = np.random.default_rng(7)
    for sh in [(n, n, n) for n in (32, 64, 96, 160, 256)]:
        ev = _evaluator(space, sh, 11)
        for g in rng.permutation(len(space.all_genomes()))[:60]:
            db.add(ev(space.all_genomes()[g]))
    target = (512, 512, 512)
    base = _evaluator(space, target, 5)

    class Bench:
        def __init__(self):
            self.space = space

        def __call__(self, g):
            clock.t += 0.1
            return base(g)

    class TimedMLP(NumpyMLP):
        def train(self, X, t, epochs, lr):
            clock.t += 0.3 * epochs / 800
            return super().train(X, t, min(epochs, 200), lr)

    out = T.study(db, target, seeds=3, ga_evals=60, bench=Bench(),
                  mlp_factory=lambda s: (lambda d: TimedMLP(d, 16, s)), clock=clock,
                  log=lambda *_: None)
    assert out["summary"]["seeds"] == 3 and len(out["runs"]) == 3
    for r in out["runs"]:
        assert r["plain_W"]["evals"] == 60 and abs(r["W"] - 6.0) < 1e-9
        for arm in ("plain_frac", "model_frac"):
            assert r[arm]["seconds"] <= 0.25 * r["W"] + 1e-9, (arm, r[arm]["seconds"])
        # the model arm paid for its training: fewer benchmarks than the plain one
        assert r["model_frac"]["evals"] < r["plain_frac"]["evals"]
    s = out["summary"]
    for arm in ("plain_W", "plain_frac", "model_frac"):
        assert s[arm]["best_mean"] > 0 and s[arm]["best_sd"] >= 0
    truth = max(synthetic_cups(space, g, target) for g in space.all_genomes())
    assert s["model_frac"]["best_mean"] >= 0.97 * truth


def test_draw_survives_tiny_spreads():
    """With spreads far below the score differences every weight but the top's underflows in a
    direct evaluation; a draw that excludes the top must still return a parent (the one with
    the largest weight)."""
    space = T.Space(3)
    ev = T.Evolution(space, np.random.default_rng(0))
    gs = space.all_genomes()[:4]
    for i, g in enumerate(gs):
        ev.scores[g] = (20e9 - 1e9 * i, 1e3)  # 1 G apart, spreads of 1 k
    top, _ = ev.top()
    picks = {ev.draw(2e3, exclude=(top,)) for _ in range(20)}
    assert picks == {gs[1]}
