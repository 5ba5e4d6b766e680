"""Independent restatement of the library's compaction order, shared by the GPU test of the
compaction pass and the CPU tests of the multi-GPU sharding (test helper, not a test)."""
import numpy as np


def expected_active_order(w):
    """Independent restatement of the compaction rule: points that pass the metadata checks,
    costliest (grid, stored-species) class first by pair count n(n+1)/2 ns + ns(ns-1)/2 n^2
    (ties: lower grid, then fewer species), ascending point index inside a class."""
    S = w.n_species
    classes = []
    for g, n in enumerate(w.bins_per_grid):
        for ns in range(1, S + 1):
            classes.append((-(ns * n * (n + 1) / 2 + ns * (ns - 1) / 2 * n * n), g, ns))
    rank = {(g, ns): r for r, (_, g, ns) in enumerate(sorted(classes, key=lambda c: c[0]))}
    keyed = []
    for p in range(w.n_points):
        if w.cloudy is not None and w.cloudy[p] == 0:
            continue
        if w.temperature is not None and not (float(w.temperature[p]) > w.t_min_K):
            continue
        ns = bin(int(w.species_mask[p])).count("1")
        if ns == 0:
            continue
        keyed.append((rank[(int(w.grid_id[p]), ns)], p))
    return np.array([p for _, p in sorted(keyed)], np.int32)
