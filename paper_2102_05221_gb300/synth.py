"""Seeded synthetic time-series inputs shaped like the paper's workloads.

The paper measures on the UCR archive (85 datasets, Section 5.1) and on the
UCR-suite sub-sequence data (Section 5.3); neither is available here, so these
generators stand in for them.  Every series is a z-normalised Gaussian random
walk (step sigma = 1), optionally plus a class template
``sin(2*pi*f_k*t/L)`` with ``f_k = k + 1`` cycles, then z-normalised again
(population standard deviation, epsilon-guarded).

This module holds no arithmetic of the elastic distances: it only draws
inputs.  Both the CUDA path's tests/bench and the CPU oracle's tests take their
inputs from here, so the two never share anything else.

Packed ("ragged") sets follow the C-ABI layout: one float32 buffer holding the
series back to back, ``int64 offsets[n]`` (element offset of each series) and
``int32 lengths[n]``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 2102_05221
_EPS = 1e-8


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def znorm(x: np.ndarray) -> np.ndarray:
    """z-normalise the last axis (population std, epsilon-guarded)."""
    x = np.asarray(x, dtype=np.float64)
    mu = x.mean(axis=-1, keepdims=True)
    sd = x.std(axis=-1, keepdims=True)
    return (x - mu) / np.maximum(sd, _EPS)


def random_walks(rng: np.random.Generator, n: int, length: int) -> np.ndarray:
    """n z-normalised Gaussian random walks of the given length (float64)."""
    if n == 0:
        return np.zeros((0, length))
    return znorm(np.cumsum(rng.standard_normal((n, length)), axis=-1))


def labelled_series(rng: np.random.Generator, labels: np.ndarray, length: int) -> np.ndarray:
    """Random walk + sine template of frequency (label+1) cycles, z-normalised."""
    walks = random_walks(rng, len(labels), length)
    tt = np.arange(length, dtype=np.float64)
    tmpl = np.sin(2.0 * math.pi * (labels[:, None] + 1.0) * tt[None, :] / length)
    return znorm(walks + tmpl).astype(np.float32)


@dataclasses.dataclass
class Dataset:
    """A train/test split of equal-length labelled series (float32, row-major)."""

    train: np.ndarray
    test: np.ndarray
    train_labels: np.ndarray
    test_labels: np.ndarray
    seed: int


def make_dataset(n_train: int, n_test: int, length: int, n_classes: int, seed: int,
                 template: bool = True) -> Dataset:
    """Train and test draws come from separate sub-streams of ``seed``."""
    c_tr, c_te = np.random.SeedSequence(seed).spawn(2)
    r_tr = np.random.Generator(np.random.PCG64(c_tr))
    r_te = np.random.Generator(np.random.PCG64(c_te))
    y_tr = r_tr.integers(0, n_classes, size=n_train)
    y_te = r_te.integers(0, n_classes, size=n_test)
    if template:
        x_tr = labelled_series(r_tr, y_tr, length)
        x_te = labelled_series(r_te, y_te, length)
    else:
        x_tr = random_walks(r_tr, n_train, length).astype(np.float32)
        x_te = random_walks(r_te, n_test, length).astype(np.float32)
    return Dataset(x_tr, x_te, y_tr.astype(np.int32), y_te.astype(np.int32), seed)


# --------------------------------------------------------------------------
# Ragged (packed) sets: float32 data + int64 offsets + int32 lengths.
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Packed:
    data: np.ndarray      # float32 [sum(lengths)]
    offsets: np.ndarray   # int64 [n]
    lengths: np.ndarray   # int32 [n]

    @property
    def count(self) -> int:
        return int(self.lengths.shape[0])

    def series(self, i: int) -> np.ndarray:
        o = int(self.offsets[i])
        return self.data[o:o + int(self.lengths[i])]

    def max_length(self) -> int:
        return int(self.lengths.max()) if self.count else 0


def pack(series_list) -> Packed:
    """Pack a list of 1-D arrays (or a 2-D array) into the ragged layout."""
    rows = [np.asarray(s, dtype=np.float32).ravel() for s in series_list]
    lengths = np.array([len(r) for r in rows], dtype=np.int32)
    offsets = np.zeros(len(rows), dtype=np.int64)
    if len(rows) > 1:
        offsets[1:] = np.cumsum(lengths[:-1], dtype=np.int64)
    data = np.concatenate(rows).astype(np.float32) if rows else np.zeros(0, np.float32)
    return Packed(data, offsets, lengths)


def ragged_walks(n: int, lengths, seed: int, n_classes: int = 0) -> Packed:
    """n series with the given lengths (array or (lo, hi) log-uniform range)."""
    rng = _rng(seed)
    if isinstance(lengths, tuple):
        lo, hi = lengths
        lens = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))).astype(int)
        lens = np.clip(lens, lo, hi)
    else:
        lens = np.asarray(lengths, dtype=int)
    out = []
    for L in lens:
        if n_classes > 0:
            y = rng.integers(0, n_classes, size=1)
            out.append(labelled_series(rng, y, int(L))[0])
        else:
            out.append(random_walks(rng, 1, int(L))[0].astype(np.float32))
    return pack(out)


def uniform_values(n: int, lengths, seed: int, lo: float = -3.0, hi: float = 3.0) -> Packed:
    """Series of i.i.d. uniform values (used for small edge-case tests)."""
    rng = _rng(seed)
    return pack([rng.uniform(lo, hi, size=int(L)).astype(np.float32) for L in lengths])


# --------------------------------------------------------------------------
# The five workload shapes (configuration recipes; sizes are the workloads').
# --------------------------------------------------------------------------

def long_series(n: int, seed: int, seg=(200, 2000), n_classes: int = 10) -> np.ndarray:
    """A long series standing in for the references of sub-sequence search
    (Section 5.3): back-to-back segments of log-uniform length in `seg`, each
    a z-normalised random walk plus a class sine template (values O(1))."""
    rng = _rng(seed)
    lo, hi = seg
    out, total = [], 0
    while total < n:
        L = int(np.clip(np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi)))), lo, hi))
        y = rng.integers(0, n_classes, size=1)
        out.append(labelled_series(rng, y, L)[0])
        total += L
    return np.concatenate(out)[:n].astype(np.float32)


def subseq_queries(T: np.ndarray, lengths, seed: int, planted: bool = True, noise: float = 0.1):
    """Queries for sub-sequence search: a window of T at a random position
    plus N(0, noise) (planted), or an independent labelled series.  Returns
    (Packed, positions) with position -1 for queries that were not planted."""
    rng = _rng(seed)
    out, where = [], []
    for m in lengths:
        m = int(m)
        if planted and m <= len(T):
            p = int(rng.integers(0, len(T) - m + 1))
            out.append((T[p:p + m] + rng.normal(0.0, noise, m)).astype(np.float32))
            where.append(p)
        else:
            y = rng.integers(0, 10, size=1)
            out.append(labelled_series(rng, y, m)[0])
            where.append(-1)
    return pack(out), np.asarray(where, dtype=np.int64)


def seed_for(config: int, dataset: int = 0) -> int:
    return BASE_SEED + config * 1000 + dataset


def workload_small_dtw(seed_offset: int = 0) -> Dataset:
    """64 train x 32 test, length 128, 4 classes (plain unpruned DTW 1-NN)."""
    return make_dataset(64, 32, 128, 4, seed_for(1, seed_offset))


def workload_nn1_512(n_train: int = 1000, n_test: int = 1000, seed_offset: int = 0) -> Dataset:
    """1000 train x 1000 test, length 512, 10 classes (EAPruned 1-NN, six distances)."""
    return make_dataset(n_train, n_test, 512, 10, seed_for(2, seed_offset))


def workload_nn1_8192(n_train: int = 200, n_test: int = 16, seed_offset: int = 0) -> Dataset:
    """200 train x 16 test, length 8192 (the longest serving set), 10 classes:
    1-NN over long series, which run one CTA per pair."""
    return make_dataset(n_train, n_test, 8192, 10, seed_for(6, seed_offset))


def workload_allpairs_4096(n: int = 256, length: int = 4096, seed_offset: int = 0) -> np.ndarray:
    """n random walks (no template) of the given length, for all-pairs matrices."""
    rng = _rng(seed_for(3, seed_offset))
    return random_walks(rng, n, length).astype(np.float32)


@dataclasses.dataclass
class UnevenDataset:
    length: int
    n_classes: int
    window_ratio: float
    data: Dataset


def workload_uneven(n_datasets: int = 64, seed_offset: int = 0,
                    len_range=(24, 2048), train_range=(16, 2000), test_range=(16, 1000),
                    class_range=(2, 20), window_range=(0.05, 0.20)) -> list:
    """64 datasets: length log-uniform in [24, 2048], train log-uniform in
    [16, 2000], test log-uniform in [16, 1000], classes uniform in {2..20},
    CDTW window ratio uniform in [5%, 20%]."""
    rng = _rng(seed_for(4, seed_offset))
    out = []
    for d in range(n_datasets):
        def lu(lo, hi):
            return int(np.clip(np.rint(math.exp(rng.uniform(math.log(lo), math.log(hi)))), lo, hi))
        L = lu(*len_range)
        ntr = lu(*train_range)
        nte = lu(*test_range)
        k = int(rng.integers(class_range[0], class_range[1] + 1))
        wr = float(rng.uniform(*window_range))
        out.append(UnevenDataset(L, k, wr, make_dataset(ntr, nte, L, k, seed_for(4, 100 + d + seed_offset))))
    return out


def serving_refsets(sizes=None, seed_offset: int = 0):
    """Resident reference sets for the serving loop: lengths 128..8192 plus a
    mixed 64..1024 set of z-normalised random walks."""
    if sizes is None:
        sizes = {128: 50000, 256: 30000, 512: 20000, 1024: 10000, 2048: 5000,
                 4096: 3000, 8192: 2000, "mixed": 20000}
    out = {}
    for i, (L, n) in enumerate(sizes.items()):
        if L == "mixed":
            out[L] = ragged_walks(n, (64, 1024), seed_for(5, 50 + i + seed_offset))
        else:
            rng = _rng(seed_for(5, i + seed_offset))
            out[L] = pack(random_walks(rng, n, int(L)).astype(np.float32))
    return out
