"""Helpers for the GPU parity tests: oracle runs and error measures."""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np

from oracle import fields, noise
from tests.oracle_cases import cosmology_from


def oracle_noise_parallel(seed, n, workers=None):
    """The oracle's W grid, its cells split over a spawn-started process pool."""
    total = n ** 3
    workers = workers or max(1, min(16, len(os.sched_getaffinity(0))))
    if total < (1 << 22) or workers == 1:
        return noise.white_noise(seed, n)
    bounds = np.linspace(0, total, 4 * workers + 1).astype(np.int64)
    out = np.empty(total, dtype=np.float64)
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
        futs = {ex.submit(_chunk, seed, int(a), int(b)): (a, b) for a, b in zip(bounds[:-1], bounds[1:])}
        for f in cf.as_completed(futs):
            a, b = futs[f]
            out[a:b] = f.result()
    return out.reshape(n, n, n)


def _chunk(seed, a, b):
    return noise.noise_at(seed, np.arange(a, b, dtype=np.int64))


def run_oracle(w, seed=None, noise_grid=None, components=(0, 1, 2), want_delta=False,
               corner=False):
    c = cosmology_from(w["cosmo"])
    if noise_grid is None and seed is not None and w["n"] >= 256:
        noise_grid = oracle_noise_parallel(seed, w["n"])
    return fields.zeldovich(w["n"], w["box"], c, w["z_init"], seed=seed, noise=noise_grid,
                            q_offset=0.0 if corner else 0.5, want_delta=want_delta,
                            components=components)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def min_image(d, box):
    return d - box * np.round(d / box)
