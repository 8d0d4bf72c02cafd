"""View sampling of the LM steps (Sec. 4.3) -- test infrastructure.

Plain Python in FP64 (sequential sums, so the results can be compared bit
for bit), written from the paper's description:

* every camera c_i gets the feature f_i = [x, y, z, dx, dy, dz]: its
  normalised location and its viewing direction.  Reading: locations are
  centred on their mean and divided by the largest distance from it (the
  unit ball); the direction is the camera's +z axis in world space;
* K-Means partitions the cameras into as many clusters as views per step
  (Lloyd's algorithm, k-means++ initialisation; ties go to the lower index,
  an emptied cluster keeps its centre, at most 100 iterations or until no
  assignment changes);
* each step takes one camera uniformly at random from every cluster.

Random numbers come from SplitMix64 (Steele, Lea, Flood 2014), keyed by
(seed, step, stream); the uniform mode (views drawn without replacement)
uses the same generator.
"""
from __future__ import annotations

import math

M64 = (1 << 64) - 1


class SplitMix64:
    """The published generator: state += golden gamma, then the two
    xor-shift-multiply rounds of the finaliser."""

    def __init__(self, state):
        self.state = state & M64

    def next(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        return z ^ (z >> 31)

    def unit(self):
        """Uniform in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / 9007199254740992.0)


def step_generator(seed, step, stream):
    """The generator of draw `stream` of LM step `step` (step -1: set-up)."""
    a = SplitMix64(seed).next()
    b = SplitMix64(a ^ ((0xD1B54A32D192ED03 * ((step + 1) & M64)) & M64)).next()
    c = SplitMix64(b ^ ((0x8CB92BA72F3D8DD7 * (stream + 1)) & M64)).next()
    return SplitMix64(c)


def uniform_views(n_cams, n_views, seed, step):
    """n_views distinct camera indices (partial Fisher-Yates), sorted."""
    k = n_cams if (n_views <= 0 or n_views >= n_cams) else n_views
    perm = list(range(n_cams))
    g = step_generator(seed, step, 0)
    if k < n_cams:
        for i in range(k):
            r = i + int(math.floor(g.unit() * (n_cams - i)))
            perm[i], perm[r] = perm[r], perm[i]
    return sorted(perm[:k])


def camera_features(world_to_cam):
    """world_to_cam: list of 12 floats per camera (row-major [R | t]).
    Returns one 6-vector per camera."""
    n = len(world_to_cam)
    pos = []
    mean = [0.0, 0.0, 0.0]
    for w in world_to_cam:
        c = []
        for a in range(3):
            v = 0.0
            for r in range(3):
                v -= float(w[4 * r + a]) * float(w[4 * r + 3])  # centre = -R^T t
            c.append(v)
            mean[a] += v
        pos.append(c)
    mean = [m / n for m in mean]
    rmax = 0.0
    for c in pos:
        d2 = 0.0
        for a in range(3):
            d = c[a] - mean[a]
            d2 += d * d
        rmax = max(rmax, math.sqrt(d2))
    feats = []
    for c, w in zip(pos, world_to_cam):
        f = [(c[a] - mean[a]) / rmax if rmax > 0.0 else 0.0 for a in range(3)]
        f += [float(w[8 + a]) for a in range(3)]  # third row of R: the +z axis in world space
        feats.append(f)
    return feats


def _d2(a, b):
    s = 0.0
    for j in range(6):
        d = a[j] - b[j]
        s += d * d
    return s


def kmeans(feats, k, seed):
    """Lloyd's algorithm with k-means++ initialisation.  Returns (labels,
    iterations)."""
    n = len(feats)
    k = min(k, n)
    g = step_generator(seed, -1, 1)
    first = min(n - 1, int(math.floor(g.unit() * n)))
    cen = [list(feats[first])]
    d2 = [_d2(f, cen[0]) for f in feats]
    for c in range(1, k):
        tot = 0.0
        for v in d2:
            tot += v
        if tot > 0.0:
            thr = g.unit() * tot
            run, pick = 0.0, n - 1
            for i, v in enumerate(d2):
                run += v
                if run > thr:
                    pick = i
                    break
        else:
            pick = c % n
        cen.append(list(feats[pick]))
        d2 = [min(d2[i], _d2(feats[i], cen[c])) for i in range(n)]
    labels = [-1] * n
    iters = 0
    for it in range(100):
        changed = False
        for i, f in enumerate(feats):
            best, bd = 0, _d2(f, cen[0])
            for c in range(1, k):
                d = _d2(f, cen[c])
                if d < bd:
                    bd, best = d, c
            if labels[i] != best:
                labels[i] = best
                changed = True
        iters = it + 1
        if not changed:
            break
        sums = [[0.0] * 6 for _ in range(k)]
        cnt = [0] * k
        for i, f in enumerate(feats):
            cnt[labels[i]] += 1
            for j in range(6):
                sums[labels[i]][j] += f[j]
        for c in range(k):
            if cnt[c] > 0:
                cen[c] = [sums[c][j] / cnt[c] for j in range(6)]
    return labels, iters


def cluster_draw(labels, k, seed, step):
    """One camera uniformly from every (non-empty) cluster, sorted."""
    members = [[] for _ in range(k)]
    for i, c in enumerate(labels):
        members[c].append(i)
    out = []
    for c in range(k):
        m = members[c]
        if not m:
            continue
        g = step_generator(seed, step, 2 + c)
        out.append(m[min(len(m) - 1, int(math.floor(g.unit() * len(m))))])
    return sorted(out)
