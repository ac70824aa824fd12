"""Lloyd k-means and the multi-level partition tree (oracle; test infrastructure only).

Sec. 3 ("Index Structure"): the base vectors are split into disjoint partitions
by k-means, each with a centroid; the centroids are clustered the same way to
make the next level.  The paper names only "k-means", so these readings are
fixed here (and identically, but independently, in the library):

  seeding   K distinct row indices by a partial Fisher-Yates shuffle driven by
            SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): state <- state + gamma;
            output = mix(state).  Step i draws z and swaps perm[i] with
            perm[i + z mod (n - i)].
  assign    argmin_c ||x - c||^2, ties to the lower centroid index.
  update    FP64 mean of the members, rounded once to FP32; an empty cluster
            keeps its previous centroid.
  stop      a fixed number of iterations.
  members   after the last update every row goes to its nearest final centroid.
  seeds     leaves use `seed`, parents use `seed + 1`.
"""

import numpy as np

from .knn import L2, distances_bulk

MASK64 = (1 << 64) - 1
SM_GAMMA = 0x9E3779B97F4A7C15
SM_MUL1 = 0xBF58476D1CE4E5B9
SM_MUL2 = 0x94D049BB133111EB


def splitmix64_next(state):
    """One SplitMix64 step: returns (new_state, 64-bit output)."""
    state = (state + SM_GAMMA) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * SM_MUL1) & MASK64
    z = ((z ^ (z >> 27)) * SM_MUL2) & MASK64
    return state, z ^ (z >> 31)


def init_rows(n, K, seed):
    """K distinct row indices in [0, n) by the seeded partial Fisher-Yates shuffle."""
    if K > n:
        raise ValueError("K > n")
    perm = np.arange(n, dtype=np.int64)
    state = seed & MASK64
    for i in range(K):
        state, z = splitmix64_next(state)
        j = i + int(z % (n - i))
        perm[i], perm[j] = perm[j], perm[i]
    return perm[:K].copy()


def assign(X, C, chunk=4096):
    """Index of the nearest centroid for every row (ties to the lower index)."""
    X = np.asarray(X)
    out = np.empty(X.shape[0], dtype=np.int64)
    for s in range(0, X.shape[0], chunk):
        D = distances_bulk(X[s:s + chunk], C, L2)
        out[s:s + chunk] = np.argmin(D, axis=1)  # first minimum = lowest index
    return out


def update(X, a, C_prev):
    """New centroids: FP64 member means rounded to FP32; empty clusters keep theirs."""
    K, d = C_prev.shape
    X = np.asarray(X)
    sums = np.empty((K, d), dtype=np.float64)
    for j in range(d):   # per-dimension FP64 sums over the members, in row order
        sums[:, j] = np.bincount(a, weights=X[:, j].astype(np.float64), minlength=K)
    counts = np.bincount(a, minlength=K)
    C = np.array(C_prev, dtype=np.float32, copy=True)
    nz = counts > 0
    C[nz] = (sums[nz] / counts[nz, None]).astype(np.float32)
    return C, counts


def lloyd(X, K, iters, seed, C0=None):
    """Lloyd iterations from the seeded initial rows (or from C0 when given)."""
    X = np.asarray(X, dtype=np.float32)
    if C0 is None:
        C = X[init_rows(X.shape[0], K, seed)].copy()
    else:
        C = np.array(C0, dtype=np.float32, copy=True)
    for _ in range(iters):
        a = assign(X, C)
        C, _ = update(X, a, C)
    return C


def objective(X, C, a):
    """Sum of squared distances of rows to their assigned centroids (FP64)."""
    diff = np.asarray(X, np.float64) - np.asarray(C, np.float64)[a]
    return float((diff * diff).sum())


class Level:
    """One level of the tree: partition centroids plus member rows and ids."""

    def __init__(self, centroids, vectors, ids):
        self.centroids = np.asarray(centroids, dtype=np.float32)
        self.vectors = [np.asarray(v, dtype=np.float32) for v in vectors]
        self.ids = [np.asarray(i, dtype=np.int64) for i in ids]

    @property
    def n_part(self):
        return self.centroids.shape[0]

    def sizes(self):
        return np.array([v.shape[0] for v in self.vectors], dtype=np.int64)


def partition_level(rows, ids, centroids):
    """Group rows by nearest centroid (members in ascending row order)."""
    a = assign(rows, centroids)
    vecs, pids = [], []
    for j in range(centroids.shape[0]):
        m = np.nonzero(a == j)[0]
        vecs.append(rows[m])
        pids.append(ids[m])
    return Level(centroids, vecs, pids), a


def build_index(X, ids, n_leaf, n_parent=0, iters=10, seed=0):
    """Multi-level index of Sec. 3: leaves = k-means(X), parents = k-means(leaf centroids).

    Returns a list of levels, level 0 first.  Level 1 (when n_parent > 0)
    holds the leaf centroids as its "vectors", with the leaf index as id.
    The top of the tree is the single partition of the last level's centroids.
    """
    X = np.asarray(X, dtype=np.float32)
    ids = np.asarray(ids, dtype=np.int64)
    C0 = lloyd(X, n_leaf, iters, seed)
    lv0, _ = partition_level(X, ids, C0)
    levels = [lv0]
    if n_parent:
        C1 = lloyd(C0, n_parent, iters, seed + 1)
        lv1, _ = partition_level(C0, np.arange(n_leaf, dtype=np.int64), C1)
        levels.append(lv1)
    return levels


def index_from_assignment(X, ids, C0, a0, C1=None, a1=None):
    """Levels from given centroids and assignments (lets tests fix the structure)."""
    X = np.asarray(X, dtype=np.float32)
    ids = np.asarray(ids, dtype=np.int64)
    C0 = np.asarray(C0, dtype=np.float32)
    lv0 = Level(C0, [X[a0 == j] for j in range(C0.shape[0])],
                [ids[a0 == j] for j in range(C0.shape[0])])
    levels = [lv0]
    if C1 is not None:
        C1 = np.asarray(C1, dtype=np.float32)
        leaf = np.arange(C0.shape[0], dtype=np.int64)
        levels.append(Level(C1, [C0[a1 == j] for j in range(C1.shape[0])],
                            [leaf[a1 == j] for j in range(C1.shape[0])]))
    return levels
