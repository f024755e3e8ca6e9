"""Pins of the oracle's tree, lists and expansion orders (Sec. 6.1-6.3).

* the Lipschitz limits printed in Sec. 6.3 (tests/golden/lipschitz_limits.txt)
  follow from Eqs. nterms_criteria_2d / nterms_criteria_3d;
* the term count of the real Laplace criterion (Eq. nterms_criteria) has a
  closed form;
* Morton prefixes equal the box coordinates floor((x - lo) 2^l / W);
* Lists 1-4 equal a brute-force O(B^2) classification from their
  definitions, and every (target leaf, source leaf) pair is covered by
  exactly one interaction path (P2P, M2L at some ancestor pair, M2P, P2L);
* the level restriction holds.
"""
import math
import os

import numpy as np
import pytest

from cfmm_inputs import curve2d, surface3d
from oracle import tree as tr

GOLD = os.path.join(os.path.dirname(__file__), "golden", "lipschitz_limits.txt")


def test_printed_lipschitz_limits():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    assert rows
    for dim, k, lmax in rows:
        f = tr.lipschitz_limit_2d if dim == "2" else tr.lipschitz_limit_3d
        assert round(f(int(k)), 4) == float(lmax)


def test_zc_matches_3d_limit_formula():
    # Lemma 5.1.1's z_c at c = R/r equals the criterion's C_L < c solution
    for k in (1, 2, 3):
        c = (k + 0.5) / (math.sqrt(3) / 2)
        assert abs(tr.z_c(c) - tr.lipschitz_limit_3d(k)) < 1e-12


@pytest.mark.parametrize("dim,k,eps", [(2, 1, 1e-6), (2, 2, 1e-9), (3, 1, 1e-6), (3, 2, 1e-3)])
def test_laplace_nterms_closed_form(dim, k, eps):
    ratio = math.sqrt(dim) / 2 / (k + 0.5)
    expect = math.ceil(math.log(eps) / math.log(ratio))
    assert tr.nterms_laplace(dim, k, eps) == expect
    if (dim, k, eps) == (2, 1, 1e-6):
        assert expect == 19


@pytest.mark.parametrize("dim", [2, 3])
def test_morton_prefix_is_box_coordinate(dim):
    rng = np.random.default_rng(3)
    re = rng.uniform(-5, 7, size=(500, dim))
    B = tr.bits_for_dim(dim)
    lo, W = tr.root_box(re)
    keys = tr.morton(tr.quantize(re, lo, W, B), B)
    for level in (1, 2, 5, 9):
        box = np.floor((re - lo) / (W / 2 ** level)).astype(np.int64)
        pre = keys >> np.uint64(dim * (B - level))
        for i in range(0, 500, 37):
            assert tr.decode(int(pre[i]), level, dim) == tuple(box[i])


def _ancestors(T, b):
    out = []
    while b >= 0:
        out.append(b)
        b = int(T.box_parent[b])
    return out


def _brute_lists(T):
    nb, k, l0 = T.nboxes, T.k, T.l0
    co = [T.coords(b) for b in range(nb)]
    lv = T.box_level
    L = {n: [[] for _ in range(nb)] for n in ("list1", "list2", "list3", "list4")}
    nr = lambda a, b: tr.near(int(lv[a]), co[a], int(lv[b]), co[b], k)
    for b in range(nb):
        if lv[b] < l0:
            continue
        for c in range(nb):
            if T.box_leaf[b] and T.box_leaf[c] and nr(b, c):
                L["list1"][b].append(c)
            if lv[c] == lv[b] and not nr(b, c):
                if lv[b] == l0 or nr(int(T.box_parent[b]), int(T.box_parent[c])):
                    L["list2"][b].append(c)
            if T.box_leaf[b] and lv[c] > lv[b] and not nr(b, c) and nr(b, int(T.box_parent[c])):
                L["list3"][b].append(c)
    for b in range(nb):
        for c in L["list3"][b]:
            L["list4"][c].append(b)
    return L


CASES = [
    dict(dim=2, n=400, N_s=4, k=1, helm=False, kappa=0.0),
    dict(dim=2, n=400, N_s=6, k=2, helm=False, kappa=0.0),
    dict(dim=2, n=600, N_s=8, k=1, helm=True, kappa=30.0),
    dict(dim=3, n=500, N_s=6, k=1, helm=False, kappa=0.0),
]


def _geom(c):
    if c["dim"] == 2:
        return curve2d(c["n"], seed=5, t_half=6.0, height=0.8)
    return surface3d(c["n"], seed=5, half=3.0, amp=0.5, width=1.0, slope=0.3, rho0=1.0)


@pytest.mark.parametrize("case", CASES)
def test_lists_match_brute_force(case):
    g = _geom(case)
    T = tr.build_tree(g.re, g.im, case["N_s"], k=case["k"], kappa=case["kappa"],
                      eps=1e-6, helmholtz=case["helm"])
    assert T.nboxes > 20
    bl = _brute_lists(T)
    for name in bl:
        for b in range(T.nboxes):
            assert sorted(bl[name][b]) == T.lists[name][b], (name, b)


@pytest.mark.parametrize("case", CASES)
def test_interaction_partition(case):
    g = _geom(case)
    T = tr.build_tree(g.re, g.im, case["N_s"], k=case["k"], kappa=case["kappa"],
                      eps=1e-6, helmholtz=case["helm"])
    leaves = [b for b in range(T.nboxes) if T.box_leaf[b]]
    l0 = T.l0
    L1 = [set(x) for x in T.lists["list1"]]
    L2 = [set(x) for x in T.lists["list2"]]
    L3 = [set(x) for x in T.lists["list3"]]
    L4 = [set(x) for x in T.lists["list4"]]
    anc = {b: [a for a in _ancestors(T, b) if T.box_level[a] >= l0] for b in leaves}
    for t in leaves:
        for s in leaves:
            cnt = int(s in L1[t])
            cnt += sum(1 for A in anc[t] for Bx in anc[s] if Bx in L2[A])
            cnt += sum(1 for Bx in anc[s] if Bx in L3[t])
            cnt += sum(1 for A in anc[t] if s in L4[A])
            assert cnt == 1, (t, s, cnt)


@pytest.mark.parametrize("case", CASES)
def test_level_restriction(case):
    g = _geom(case)
    T = tr.build_tree(g.re, g.im, case["N_s"], k=case["k"], kappa=case["kappa"],
                      eps=1e-6, helmholtz=case["helm"])
    assert tr.check_balance(T)
    # every leaf holds <= N_s points unless it sits at the deepest level
    for b in range(T.nboxes):
        if T.box_leaf[b]:
            assert T.box_end[b] - T.box_start[b] <= T.N_s or T.box_level[b] == T.B
    # the leaves partition the sorted points
    cover = np.zeros(len(g.re), int)
    for b in range(T.nboxes):
        if T.box_leaf[b]:
            cover[T.box_start[b]:T.box_end[b]] += 1
    assert np.all(cover == 1)


def test_top_level_rule_helmholtz():
    g = curve2d(3000, seed=3, t_half=10.0, height=0.5)
    T = tr.build_tree(g.re, g.im, 32, k=1, kappa=20.0, eps=1e-6, helmholtz=True)
    tau = tr.C_TOP[2] * math.log(1e-6 / tr.EPS_MACH)
    im = g.im[T.perm]

    def spread(b):
        seg = im[T.box_start[b]:T.box_end[b]]
        return 20.0 * math.sqrt(2) * np.max(seg.max(0) - seg.min(0))
    # at l0 every box satisfies the spread bound; one level up some box does not
    for b in range(T.level_offset[T.l0], T.level_offset[T.l0 + 1]):
        assert spread(b) <= tau
    assert max(spread(b) for b in range(T.level_offset[T.l0 - 1], T.level_offset[T.l0])) > tau
    assert T.l0 >= 2
    # no leaf above l0
    assert np.all(T.box_level[T.box_leaf] >= T.l0)


# ---- the "near" predicate of Sec. 6.2 pinned by counts fixed by the definitions ----

@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_near_colleague_count_interior(dim, k):
    """Same-level boxes are near exactly when they are k-colleagues: an interior
    box has (2k+1)^d of them (itself included)."""
    level = 4
    I = tuple([8] * dim)
    cnt = sum(tr.near(level, I, level, J, k) for J in np.ndindex(*([1 << level] * dim)))
    assert cnt == (2 * k + 1) ** dim


def test_near_boundary_hand_cases():
    """Boxes of different levels: near means ||c_a - c_b||_inf <= k/2 (w_a + w_b),
    with equality (touching boxes at k = 1) counting as near. Level-1 box (0, 0)
    spans [0, 1/2]^2 (centre 1/4, width 1/2); level-2 box (2, 0) spans
    [1/2, 3/4] x [0, 1/4] (centre 5/8): distance 3/8 = (1/2)(1/2 + 1/4)."""
    assert tr.near(1, (0, 0), 2, (2, 0), 1)
    assert tr.near(2, (2, 0), 1, (0, 0), 1)
    # level-2 box (3, 0): centre 7/8, distance 5/8 > 3/8, but <= 2/2 (3/4) at k = 2
    assert not tr.near(1, (0, 0), 2, (3, 0), 1)
    assert tr.near(1, (0, 0), 2, (3, 0), 2)
    # level-3 box (6, 0) spans [3/4, 7/8]: centre 13/16, distance 9/16 > (1/2)(1/2 + 1/8)
    assert not tr.near(1, (0, 0), 3, (6, 0), 1)
    # level-3 box (4, 5): x touches (distance 5/16 = (1/2)(5/8)), y centre 11/16 is 7/16 away
    assert not tr.near(1, (0, 0), 3, (4, 5), 1)
    assert tr.near(1, (0, 0), 3, (4, 3), 1)
    # a diagonal neighbour at the same level touches at a corner
    assert tr.near(3, (2, 2, 2), 3, (3, 3, 3), 1)
    assert not tr.near(3, (2, 2, 2), 3, (4, 3, 3), 1)


@pytest.mark.parametrize("dim,per_axis,k,list1,list2", [(2, 16, 1, 9, 27), (2, 16, 2, 25, 75),
                                                         (3, 8, 1, 27, 189)])
def test_uniform_tree_list_sizes(dim, per_axis, k, list1, list2):
    """A complete tree (one point per finest box, leaf size 1): an interior
    leaf whose parent's colleagues all exist has (2k+1)^d List-1 leaves and
    (2(2k+1))^d - (2k+1)^d List-2 boxes (27 in 2D and 189 in 3D at k = 1)."""
    ax = np.arange(per_axis) / (per_axis - 1)
    grid = np.stack(np.meshgrid(*([ax] * dim), indexing="ij"), axis=-1).reshape(-1, dim)
    T = tr.build_tree(grid, np.zeros_like(grid), 1, k=k)
    level = int(round(math.log2(per_axis)))
    assert T.nlevels == level + 1
    assert np.sum(T.box_leaf) == per_axis ** dim
    I = tuple([per_axis // 2 - 1] * dim)
    b = T._index[(level, tr.encode(I, level, dim))]
    assert len(T.lists["list1"][b]) == list1
    assert len(T.lists["list2"][b]) == list2
    assert T.lists["list3"][b] == [] and T.lists["list4"][b] == []


# ---- Lipschitz estimate and the automatic separation (Sec. 4.1, 5.1, 6.3) ----

@pytest.mark.parametrize("slope", [0.3, 0.5, 0.8])
def test_lipschitz_estimate_curve_closed_form(slope):
    """On the curve family Im x = (phi(t), 0) with phi of slope s beyond |t| = 4
    and Re x = (t, h e^{-t^2}), |Im dx|/|Re dx| <= s, with equality (to the
    bump's e^{-16}) for pairs beyond |t| = 4."""
    g = curve2d(4000, seed=1, t_half=10.0, height=0.3, slope=slope)
    T = tr.build_tree(g.re, g.im, 32)
    L = tr.lipschitz_estimate(g.re[T.perm], g.im[T.perm])
    assert slope * (1 - 1e-9) <= L <= slope * (1 + 1e-9)


def test_lipschitz_estimate_surface_and_violation():
    g = surface3d(4000, seed=1, half=10.0, slope=0.4, rho0=3.0)
    T = tr.build_tree(g.re, g.im, 32)
    L = tr.lipschitz_estimate(g.re[T.perm], g.im[T.perm])
    assert 0.3 <= L <= 0.4 * (1 + 1e-9)
    # a slope above 1 makes Re r^2 < 0 possible: the estimate reaches 1
    g = curve2d(2000, seed=2, slope=1.3)
    T = tr.build_tree(g.re, g.im, 32)
    assert tr.lipschitz_estimate(g.re[T.perm], g.im[T.perm]) >= 1.0
    # equal real parts with different imaginary parts
    re = np.array([[0.0, 0.0], [0.0, 0.0], [1.0, 0.0]])
    im = np.array([[0.0, 0.0], [0.1, 0.0], [0.0, 0.0]])
    assert tr.lipschitz_estimate(re, im) == math.inf


def test_auto_separation_from_printed_limits():
    """With the limits printed in Sec. 6.3 (2D 0.3592, 0.5590; 3D 0.1270) and the
    factor 2: a 2D slope 0.5 keeps k = 1; the 3D surface slope 0.4 takes k = 2
    (0.254 < 0.4 <= 0.599); slope 0.73 takes k = 3; beyond every limit, k = 3."""
    assert tr.auto_separation(2, 0.5) == 1
    assert tr.auto_separation(2, 0.8) == 2
    assert tr.auto_separation(3, 0.2) == 1
    assert tr.auto_separation(3, 0.4) == 2
    assert tr.auto_separation(3, 0.73) == 3
    assert tr.auto_separation(3, 0.95) == 3
