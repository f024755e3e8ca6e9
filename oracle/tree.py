"""Tree on the real parts, level restriction, centres, Lists 1-4, expansion orders.

Test infrastructure (oracle). Follows Sec. 6.1 (tree generation on Re x,
level restriction, complexified centres Eq. complexify_center_average),
Sec. 6.2 (k-colleagues, Lists 1-4) and Sec. 6.3 (number of terms per level,
Eqs. nterms_criteria / nterms_criteria_2d / nterms_criteria_3d with the
prefactors ignored as the paper does in practice).

Readings:

* root box: centre = (min+max)/2 of Re x per axis, width W = max extent *
  (1 + 2^-20); integer coordinates q = floor((x - lo)/W * 2^B) clamped to
  [0, 2^B - 1] with B = 31 (2D) or 21 (3D); Morton key interleaves the bits
  of q with the x bit lowest. Points are ordered by a stable sort of the keys.
* a box is split when it holds more than N_s points (Sec. 6.1); empty
  children are not created; boxes at the deepest level B are never split.
* "near": boxes a, b (any levels) are near when
  ||x_a - x_b||_inf <= k/2 (w_a + w_b); at equal levels this is the
  k-colleague relation ||x_a - x_b||_inf <= k w (Sec. 6.2).
* level restriction (Sec. 6.1): a leaf may not be near any box two levels
  finer; violating leaves are split until no violation remains (the least
  fixed point, so the result does not depend on the order of splits).
  This implies the printed condition (childless boxes two or more levels
  apart are separated by more than k/2 (w1 + w2)).
* Lists (Sec. 6.2) for box b at level l:
    List 1 (leaf b): leaves c near b (b included).
    List 2: boxes c at level l, parent(c) a colleague of parent(b), c not near b;
            at the top expansion level l0, all boxes at l0 not near b.
    List 3 (leaf b): boxes c finer than b, not near b, with parent(c) near b.
    List 4: leaves a coarser than b with b in List 3 of a.
* top expansion level l0 (a departure for Helmholtz, Sec. 6.5 catastrophic
  cancellation): Laplace uses l0 = 1. Helmholtz uses the coarsest level l >= 1
  whose boxes have kappa*sqrt(d)*g_l <= tau(eps), g_l the largest per-axis
  spread of Im x inside one box of level l (a coarser leaf counts with its
  own spread), tau = c_d ln(eps/2^-52) with c_2 = 1 and c_3 = 2 (calibrated:
  on the 2D curve workload at kappa = 20 and 50, top levels three to four
  above the c = 1/4 choice gave the same errors at eps = 1e-6 and 1e-9, and
  c = 1/4 costs up to 2.6 times more; on the 3D surface workload the error
  grows with the top level like exp(0.56 kappa g), a third of the exponent
  sqrt(3) kappa g of the rule, so c_3 = 2 still bounds the growth by
  (eps/2^-52)^0.65; at kappa = 15 the level it picks met eps = 1e-6 with
  1.4e-7, at a third of the cost of the c_3 = 1 level). When no level of the
  tree qualifies (a shallow tree), the spread below the deepest level is
  taken to halve with each further level (Im x is Lipschitz in Re x, so a
  box's spread scales with its width), and l0 is the first level where that
  extrapolated spread meets the bound. Leaves above l0 are split
  down to l0 and the tree is re-balanced. M2L at l0 runs over all non-near
  pairs of l0 boxes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

EPS_MACH = 2.0 ** -52
C_TOP = {2: 1.0, 3: 2.0}   # c_d of the top-level rule (module docstring)


def bits_for_dim(dim):
    return 31 if dim == 2 else 21


def root_box(re):
    """Root square: returns (lo[dim], W)."""
    mn = re.min(axis=0)
    mx = re.max(axis=0)
    c = (mn + mx) * 0.5
    ext = float(np.max(mx - mn))
    W = ext * (1.0 + 2.0 ** -20)
    if W == 0.0:
        W = 1.0
    lo = c - W * 0.5
    return lo, W


def quantize(re, lo, W, B):
    """q = floor((x - lo)/W * 2^B), clamped (float64, no fused multiply-add)."""
    t = (re - lo[None, :]) / W
    t = t * float(2 ** B)
    q = np.floor(t)
    q = np.clip(q, 0, 2 ** B - 1).astype(np.int64)
    return q


def morton(q, B):
    """Interleave bits of q[:, d] (x bit lowest) into uint64 keys."""
    n, dim = q.shape
    key = np.zeros(n, dtype=np.uint64)
    for b in range(B):
        for d in range(dim):
            bit = ((q[:, d] >> b) & 1).astype(np.uint64)
            key |= bit << np.uint64(b * dim + d)
    return key


def decode(prefix, level, dim):
    """Integer box coordinates (tuple) of a level-`level` prefix."""
    I = [0] * dim
    for b in range(level):
        for d in range(dim):
            I[d] |= ((prefix >> (b * dim + d)) & 1) << b
    return tuple(I)


def encode(I, level, dim):
    p = 0
    for b in range(level):
        for d in range(dim):
            p |= ((I[d] >> b) & 1) << (b * dim + d)
    return p


def near(la, Ia, lb, Ib, k):
    """||x_a - x_b||_inf <= k/2 (w_a + w_b) in exact integer arithmetic."""
    m = max(la, lb)
    sa, sb = 1 << (m - la), 1 << (m - lb)
    lim = k * (sa + sb)
    for d in range(len(Ia)):
        ca = (2 * Ia[d] + 1) * sa
        cb = (2 * Ib[d] + 1) * sb
        if abs(ca - cb) > lim:
            return False
    return True


@dataclass
class Tree:
    dim: int
    B: int
    N_s: int
    k: int
    lo: np.ndarray
    W: float
    keys: np.ndarray            # sorted Morton keys (uint64)
    perm: np.ndarray            # sorted position -> input index
    leaves: list                # [(level, prefix, start, end)] in Morton order
    l0: int = 1
    # boxes, level-major, prefix-sorted inside a level
    box_level: np.ndarray = None
    box_prefix: np.ndarray = None
    box_start: np.ndarray = None
    box_end: np.ndarray = None
    box_leaf: np.ndarray = None
    box_parent: np.ndarray = None
    level_offset: np.ndarray = None
    lists: dict = field(default_factory=dict)   # name -> list of lists (per box)

    @property
    def nboxes(self):
        return len(self.box_level)

    @property
    def nlevels(self):
        return len(self.level_offset) - 1

    def coords(self, b):
        return decode(int(self.box_prefix[b]), int(self.box_level[b]), self.dim)

    def width(self, level):
        return self.W * 2.0 ** (-level)

    def real_center(self, b):
        lvl = int(self.box_level[b])
        I = self.coords(b)
        w = self.width(lvl)
        return np.array([self.lo[d] + (I[d] + 0.5) * w for d in range(self.dim)])


def _prefix(keys, level, B, dim):
    return keys >> np.uint64(dim * (B - level))


def _split_leaf(keys, B, dim, leaf):
    level, p, s, e = leaf
    sub = _prefix(keys[s:e], level + 1, B, dim).astype(np.int64)
    out = []
    for c in range(1 << dim):
        cp = (p << dim) | c
        a = s + int(np.searchsorted(sub, cp, side="left"))
        b = s + int(np.searchsorted(sub, cp, side="right"))
        if b > a:
            out.append((level + 1, cp, a, b))
    return out


def _refine(keys, B, dim, leaves, N_s, force_level):
    """Split leaves while count > N_s or level < force_level (and level < B)."""
    changed = True
    while changed:
        changed = False
        new = []
        for lf in leaves:
            level, p, s, e = lf
            if level < B and (e - s > N_s or level < force_level):
                new.extend(_split_leaf(keys, B, dim, lf))
                changed = True
            else:
                new.append(lf)
        leaves = new
    return leaves


def _box_sets(leaves, dim):
    """Per level, the set of prefixes of boxes that exist (ancestors of leaves)."""
    maxl = max(l for l, _, _, _ in leaves)
    sets = [set() for _ in range(maxl + 1)]
    for level, p, _, _ in leaves:
        for m in range(level + 1):
            sets[m].add(p >> (dim * (level - m)))
    return sets


def _violators(leaves, dim, k):
    sets = _box_sets(leaves, dim)
    maxl = len(sets) - 1
    lo_off = -((5 * k - 3) // 2)       # ceil((3 - 5k)/2)
    hi_off = (3 + 5 * k) // 2          # floor((3 + 5k)/2)
    out = []
    for i, (level, p, _, _) in enumerate(leaves):
        m = level + 2
        if m > maxl:
            continue
        I = decode(p, level, dim)
        found = False
        for off in np.ndindex(*([hi_off - lo_off + 1] * dim)):
            J = tuple(4 * I[d] + lo_off + off[d] for d in range(dim))
            if any(j < 0 or j >= (1 << m) for j in J):
                continue
            if all(0 <= J[d] - 4 * I[d] <= 3 for d in range(dim)):
                continue  # inside the leaf itself
            if encode(J, m, dim) in sets[m] and near(level, I, m, J, k):
                found = True
                break
        if found:
            out.append(i)
    return out


def _balance(keys, B, dim, leaves, k):
    while True:
        bad = set(_violators(leaves, dim, k))
        if not bad:
            return leaves
        new = []
        for i, lf in enumerate(leaves):
            if i in bad and lf[0] < B:
                new.extend(_split_leaf(keys, B, dim, lf))
            else:
                new.append(lf)
        leaves = new


def _build_boxes(T):
    dim = T.dim
    leaves = T.leaves
    maxl = max(l for l, _, _, _ in leaves)
    per_level = []
    for m in range(maxl + 1):
        d = {}
        for level, p, s, e in leaves:
            if level < m:
                continue
            q = p >> (dim * (level - m))
            if q in d:
                d[q][0] = min(d[q][0], s)
                d[q][1] = max(d[q][1], e)
                if level == m:
                    d[q][2] = True
            else:
                d[q] = [s, e, level == m]
        per_level.append(sorted(d.items()))
    lvl, pre, st, en, lf, off = [], [], [], [], [], [0]
    for m, items in enumerate(per_level):
        for q, (s, e, isleaf) in items:
            lvl.append(m)
            pre.append(q)
            st.append(s)
            en.append(e)
            lf.append(isleaf)
        off.append(len(lvl))
    T.box_level = np.array(lvl, dtype=np.int64)
    T.box_prefix = np.array(pre, dtype=np.int64)
    T.box_start = np.array(st, dtype=np.int64)
    T.box_end = np.array(en, dtype=np.int64)
    T.box_leaf = np.array(lf, dtype=bool)
    T.level_offset = np.array(off, dtype=np.int64)
    index = {}
    for b in range(len(lvl)):
        index[(lvl[b], pre[b])] = b
    T._index = index
    par = np.full(len(lvl), -1, dtype=np.int64)
    for b in range(len(lvl)):
        if lvl[b] > 0:
            par[b] = index[(lvl[b] - 1, pre[b] >> dim)]
    T.box_parent = par


def imag_spread(T, im_sorted):
    """Per box: largest per-axis range of Im x over its points (exact max/min)."""
    out = np.zeros(T.nboxes)
    for b in range(T.nboxes):
        s, e = T.box_start[b], T.box_end[b]
        seg = im_sorted[s:e]
        out[b] = float(np.max(seg.max(axis=0) - seg.min(axis=0)))
    return out


def choose_l0(T, im_sorted, kappa, eps, helmholtz):
    """Top expansion level (see module docstring)."""
    if not helmholtz:
        return 1
    tau = C_TOP[T.dim] * math.log(eps / EPS_MACH)
    g = imag_spread(T, im_sorted)
    maxl = T.nlevels - 1
    if maxl < 1:
        return 1
    sq = math.sqrt(T.dim)
    gm = 0.0
    for m in range(1, maxl + 1):
        gm = 0.0
        for b in range(T.nboxes):
            lv = T.box_level[b]
            if lv == m or (lv < m and T.box_leaf[b]):
                gm = max(gm, g[b])
        if kappa * sq * gm <= tau:
            return m
    # below the deepest level: the spread halves per level
    m = maxl
    while m < T.B and kappa * sq * gm > tau:
        m += 1
        gm *= 0.5
    return m


def build_tree(re, im, N_s, k=1, kappa=0.0, eps=1e-6, helmholtz=False, top_level=0):
    """Build the complete tree (leaves, boxes, lists) for points re/im [n][dim].

    top_level > 0 forces the top expansion level l0 instead of the rule."""
    re = np.asarray(re, dtype=np.float64)
    im = np.asarray(im, dtype=np.float64)
    n, dim = re.shape
    B = bits_for_dim(dim)
    lo, W = root_box(re)
    q = quantize(re, lo, W, B)
    keys_all = morton(q, B)
    perm = np.argsort(keys_all, kind="stable")
    keys = keys_all[perm]
    leaves = [(0, 0, 0, n)]
    leaves = _refine(keys, B, dim, leaves, N_s, 0)
    leaves = _balance(keys, B, dim, leaves, k)
    T = Tree(dim=dim, B=B, N_s=N_s, k=k, lo=lo, W=W, keys=keys, perm=perm, leaves=leaves)
    _build_boxes(T)
    im_sorted = im[perm]
    l0 = 1
    if n > N_s:
        l0 = top_level if top_level > 0 else choose_l0(T, im_sorted, kappa, eps, helmholtz)
        if l0 > 1:
            T.leaves = _balance(keys, B, dim, _refine(keys, B, dim, T.leaves, N_s, l0), k)
            _build_boxes(T)
    T.l0 = l0
    build_lists(T)
    T.center_re = np.array([T.real_center(b) for b in range(T.nboxes)]).reshape(T.nboxes, dim)
    T.center_im = np.array([im_sorted[T.box_start[b]:T.box_end[b]].sum(axis=0)
                            / (T.box_end[b] - T.box_start[b]) for b in range(T.nboxes)]).reshape(T.nboxes, dim)
    return T


def build_lists(T):
    """Lists 1-4 (module docstring), each per box sorted by box index."""
    dim, k = T.dim, T.k
    nb = T.nboxes
    l0 = T.l0
    coords = [T.coords(b) for b in range(nb)]
    lv = T.box_level
    idx = T._index
    L1 = [[] for _ in range(nb)]
    L2 = [[] for _ in range(nb)]
    L3 = [[] for _ in range(nb)]
    L4 = [[] for _ in range(nb)]
    multi = nb > 1

    def lookup(level, J):
        if level < 0 or any(j < 0 or j >= (1 << level) for j in J):
            return -1
        return idx.get((level, encode(J, level, dim)), -1)

    def colleagues(b):
        level, I = int(lv[b]), coords[b]
        out = []
        for off in np.ndindex(*([2 * k + 1] * dim)):
            J = tuple(I[d] + off[d] - k for d in range(dim))
            c = lookup(level, J)
            if c >= 0:
                out.append(c)
        return out

    def children(b):
        level, p = int(lv[b]), int(T.box_prefix[b])
        out = []
        for c in range(1 << dim):
            j = idx.get((level + 1, (p << dim) | c), -1)
            if j >= 0:
                out.append(j)
        return out

    for b in range(nb):
        level = int(lv[b])
        if not multi:
            break
        if level < l0:
            continue
        I = coords[b]
        # List 2
        if level == l0:
            for c in range(T.level_offset[level], T.level_offset[level + 1]):
                if not near(level, I, level, coords[c], k):
                    L2[b].append(c)
        else:
            for pc in colleagues(int(T.box_parent[b])):
                for c in children(pc):
                    if not near(level, I, level, coords[c], k):
                        L2[b].append(c)
        if not T.box_leaf[b]:
            continue
        # List 1 and List 3 by descending from the colleagues
        for c in colleagues(b):
            stack = [c]
            while stack:
                e = stack.pop()
                if T.box_leaf[e]:
                    L1[b].append(e)
                    continue
                for ch in children(e):
                    if near(level, I, int(lv[ch]), coords[ch], k):
                        stack.append(ch)
                    else:
                        L3[b].append(ch)
        # coarser near leaves (levels l-1 and above the colleagues)
        a = int(T.box_parent[b])
        while a >= 0:
            for c in colleagues(a):
                if T.box_leaf[c] and near(level, I, int(lv[c]), coords[c], k):
                    L1[b].append(c)
            a = int(T.box_parent[a])
    if not multi:
        L1[0].append(0)
    for b in range(nb):
        for c in L3[b]:
            L4[c].append(b)
    T.lists = {name: [sorted(set(x)) for x in L] for name, L in
               (("list1", L1), ("list2", L2), ("list3", L3), ("list4", L4))}
    # List 1 must not contain duplicates and holds only leaves
    return T


def check_balance(T):
    """True when no leaf is near a box two or more levels finer."""
    coords = [T.coords(b) for b in range(T.nboxes)]
    leaves = [b for b in range(T.nboxes) if T.box_leaf[b]]
    for b in leaves:
        for c in range(T.nboxes):
            if T.box_level[c] >= T.box_level[b] + 2 and near(
                    int(T.box_level[b]), coords[b], int(T.box_level[c]), coords[c], T.k):
                return False
    return True


# ---- expansion orders (Sec. 6.3) -----------------------------------------

# The criteria of Eqs. nterms_criteria_2d/3d are applied with the Lipschitz
# prefactor dropped, as the paper does in practice, and with headroom: the
# order is chosen for eps * P_HEADROOM (Laplace) or eps * P_HEADROOM_HELM
# (Helmholtz, whose criterion |H_n(kR) J_n(kr)| carries an extra 1/(n pi)
# against (r/R)^n and undershoots by about a digit).
P_HEADROOM = 0.1
P_HEADROOM_HELM = 0.01

def nterms_laplace(dim, k, eps):
    """Smallest n >= 1 with (r/R)^n <= eps, R=(k+1/2)w, r=sqrt(d)/2 w."""
    ratio = (math.sqrt(dim) * 0.5) / (k + 0.5)
    t = 1.0
    n = 0
    while True:
        n += 1
        t *= ratio
        if t <= eps:
            return n


def nterms_helmholtz(dim, k, eps, kappa, w, fn_pair, pmax=2000):
    """Smallest n with |f_n(kappa R) g_n(kappa r)| <= eps for n..n+3 (the Sec. 6.3
    criterion with its prefactor dropped, four consecutive orders for safety)."""
    R = (k + 0.5) * w
    r = math.sqrt(dim) * 0.5 * w
    vals = fn_pair(np.arange(pmax + 4), kappa * R, kappa * r)
    ok = np.abs(vals) <= eps
    for n in range(1, pmax):
        if ok[n] and ok[n + 1] and ok[n + 2] and ok[n + 3]:
            return n
    return pmax


def helm2d_pair(n, zR, zr):
    import scipy.special as sps
    return sps.hankel1(n, zR) * sps.jv(n, zr)


def helm3d_pair(n, zR, zr):
    import scipy.special as sps
    h = np.sqrt(np.pi / (2 * zR)) * sps.hankel1(n + 0.5, zR)
    return h * sps.spherical_jn(n, zr)


LIP_WINDOW = 32          # pairs at most this far apart in Morton order
SEP_LIP_FACTOR = 2.0     # calibrated factor of the automatic separation rule


def lipschitz_estimate(re_sorted, im_sorted):
    """Estimate of the Lipschitz constant L of Im x against Re x (Assumptions
    4.1/5.1, Eq. Lipschitz_assumption): max over pairs of points at most
    LIP_WINDOW apart in Morton order of |Im(x_i - x_j)| / |Re(x_i - x_j)|
    (inf when the real parts coincide and the imaginary parts do not; pairs
    of coincident points are skipped). L >= 1 allows Re r^2 <= 0 (Sec. 4.1),
    which the method excludes."""
    n = re_sorted.shape[0]
    best = 0.0
    for s in range(1, min(LIP_WINDOW, n - 1) + 1):
        a2 = np.sum((re_sorted[s:] - re_sorted[:-s]) ** 2, axis=1)
        b2 = np.sum((im_sorted[s:] - im_sorted[:-s]) ** 2, axis=1)
        m = b2 > 0
        if not np.any(m):
            continue
        if np.any(a2[m] == 0):
            return math.inf
        best = max(best, float(np.max(b2[m] / a2[m])))
    return math.sqrt(best)


def auto_separation(dim, L):
    """Separation for a geometry with Lipschitz estimate L: the smallest k in
    1..3 whose Sec. 6.3 limit (lipschitz_limit_2d/3d) times SEP_LIP_FACTOR is
    at least L, else 3. The factor is a calibrated reading: the criteria bound
    the worst case over all geometries, and the configurations' surfaces meet
    eps = 1e-6 at k = 2 up to slopes about twice the k = 2 limit."""
    lim = lipschitz_limit_2d if dim == 2 else lipschitz_limit_3d
    for k in (1, 2, 3):
        if SEP_LIP_FACTOR * lim(k) >= L:
            return k
    return 3


def lipschitz_limit_2d(k):
    """Largest L with ((1+L)/(1-L)) * r/R < 1, R=(k+1/2)w, r=sqrt(2)/2 w (Eq. nterms_criteria_2d)."""
    c = (k + 0.5) / (math.sqrt(2) * 0.5)
    return (c - 1.0) / (c + 1.0)


def lipschitz_limit_3d(k):
    """Largest L with C_L * r/R < 1, C_L=sqrt(L^2+10L+1)/(1-L) (Eqs. eta_const, nterms_criteria_3d)."""
    c = (k + 0.5) / (math.sqrt(3) * 0.5)
    # C_L = c  <=>  L^2 + 10L + 1 = c^2 (1-L)^2
    a = 1.0 - c * c
    bq = 10.0 + 2.0 * c * c
    cq = 1.0 - c * c
    disc = bq * bq - 4 * a * cq
    roots = [(-bq + math.sqrt(disc)) / (2 * a), (-bq - math.sqrt(disc)) / (2 * a)]
    return min(x for x in roots if 0 < x < 1)


def z_c(c):
    """Lemma 5.1.1: Lipschitz bound z_c = (c^2 + 5 - sqrt(12c^2 + 24))/(c^2 - 1)."""
    return (c * c + 5.0 - math.sqrt(12.0 * c * c + 24.0)) / (c * c - 1.0)
