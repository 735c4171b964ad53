"""Pins of the oracle's AMR tree (rules 1-7 of Sec. 3.1) by brute force on small meshes.

After random refine/coarsen flags the tree must satisfy, checked cell by cell:
  * statuses: sigma in {-1, 0, 1}; children come in complete blocks of r^d; a cell has
    children of status <= 0 iff it is a virtual mother (-1); virtual children (1) have an
    active mother (rule 2);
  * rule 4: every Voronoi neighbour of a virtual mother has children;
  * rule 5: active cells that touch (share a node) differ by at most one level, checked on
    a map of leaf levels at the finest resolution;
  * micro-patches: every active cell of level l has all cells of its (2M+1)^d box on level l;
  * refine flags on active cells below l_max are honoured; zero flags change nothing;
  * virtual children exist only where rule 4 asks for them (minimal tree).
"""
import itertools

import numpy as np
import pytest

import oracle


def tree_maps(meta, lmax, L0, d, r):
    maps = []
    for lv in range(lmax + 1):
        n = [L0[a] * r ** lv for a in range(d)] + [1] * (3 - d)
        m = np.full(n[::-1], oracle.ST_NONE, dtype=np.int8)
        maps.append(m)
    for lv, st, i, j, k in meta:
        maps[lv][k, j, i] = st
    return maps


def bc_map(c, n, periodic):
    if 0 <= c < n:
        return c, True
    if periodic:
        return c % n, True
    return min(max(c, 0), n - 1), False


def check_tree(meta, lmax, L0, d, r, M, periodic, flags=None, old_meta=None):
    maps = tree_maps(meta, lmax, L0, d, r)
    offs = [o for o in itertools.product((-1, 0, 1), repeat=d) if any(o)]
    for lv in range(lmax + 1):
        m = maps[lv]
        Z, Y, X = m.shape
        for k, j, i in itertools.product(range(Z), range(Y), range(X)):
            st = m[k, j, i]
            if st == oracle.ST_NONE:
                continue
            ijk = (i, j, k)
            # children
            if lv < lmax:
                kids = maps[lv + 1][r * k: r * k + (r if d == 3 else 1), r * j: r * j + r, r * i: r * i + r]
                exist = kids != oracle.ST_NONE
                assert exist.all() or not exist.any(), "incomplete child block"
                if st == -1:
                    assert exist.all() and np.all(kids <= 0)
                elif exist.any():
                    assert st == 0 and np.all(kids == 1)
            else:
                assert st != -1
            if lv > 0:
                ms = maps[lv - 1][k // r if d == 3 else 0, j // r, i // r]
                assert (ms == -1) if st <= 0 else (ms == 0)
            else:
                assert st in (0, -1)
            if st == -1:
                # rule 4: every Voronoi neighbour has children
                for o in offs:
                    c = []
                    ok = True
                    for a in range(d):
                        v, ins = bc_map(ijk[a] + o[a], m.shape[::-1][a], periodic)
                        ok &= ins
                        c.append(v)
                    if not ok:
                        continue
                    c += [0] * (3 - d)
                    assert m[c[2], c[1], c[0]] in (0, -1)
                    kid = maps[lv + 1][r * c[2] if d == 3 else 0, r * c[1], r * c[0]]
                    assert kid != oracle.ST_NONE, "rule 4 violated"
            if st == 1:
                # minimality: the mother has a refined Voronoi neighbour
                mm = maps[lv - 1]
                mi = [ijk[a] // r for a in range(d)]
                found = False
                for o in offs:
                    c = []
                    ok = True
                    for a in range(d):
                        v, ins = bc_map(mi[a] + o[a], mm.shape[::-1][a], periodic)
                        ok &= ins
                        c.append(v)
                    if ok:
                        c += [0] * (3 - d)
                        found |= mm[c[2], c[1], c[0]] == -1
                assert found, "superfluous virtual children"
            if st == 0 and lv > 0:
                # micro-patch: the (2M+1)^d box exists on this level
                for o in itertools.product(range(-M, M + 1), repeat=d):
                    c = [bc_map(ijk[a] + o[a], m.shape[::-1][a], periodic)[0] for a in range(d)] + [0] * (3 - d)
                    assert m[c[2], c[1], c[0]] != oracle.ST_NONE, "micro-patch incomplete"
    # rule 5 on leaves: map of leaf levels at the finest resolution
    fine = [L0[a] * r ** lmax for a in range(d)]
    leaf = np.full(fine[::-1] + [1] * (3 - d), -1, dtype=np.int32).reshape(([fine[2]] if d == 3 else [1]) + fine[:2][::-1])
    for lv, st, i, j, k in meta:
        if st != 0:
            continue
        s = r ** (lmax - lv)
        if d == 3:
            leaf[k * s:(k + 1) * s, j * s:(j + 1) * s, i * s:(i + 1) * s] = lv
        else:
            leaf[0, j * s:(j + 1) * s, i * s:(i + 1) * s] = lv
    assert np.all(leaf >= 0), "active cells must tile the domain"
    for o in offs:
        sh = [0, 0, 0]
        for a in range(d):
            sh[2 - a] = o[a]
        rolled = np.roll(leaf, shift=tuple(-x for x in sh), axis=(0, 1, 2))
        diff = np.abs(rolled - leaf)
        if not periodic:
            # ignore wrapped pairs
            sl = [slice(None)] * 3
            for ax in range(3):
                if sh[ax] == 1:
                    sl[ax] = slice(0, -1)
                elif sh[ax] == -1:
                    sl[ax] = slice(1, None)
            diff = diff[tuple(sl)]
        assert diff.max() <= 1, "rule 5 violated"
    if flags is not None and old_meta is not None:
        new = {(lv, i, j, k): st for lv, st, i, j, k in meta}
        for f, (lv, st, i, j, k) in zip(flags, old_meta):
            if f == 1 and st == 0 and lv < lmax:
                assert new[(lv, i, j, k)] == -1, "refine flag not honoured"


@pytest.mark.parametrize("d,M,lmax,periodic,seed", [
    (2, 2, 2, True, 0), (2, 3, 2, False, 1), (2, 3, 3, True, 2), (3, 2, 2, False, 3)])
def test_random_flags_keep_tree_invariants(d, M, lmax, periodic, seed):
    r = 3
    L0 = [5, 4, 3][:d]
    cfg = oracle.make_cfg(dim=d, M=M, n=tuple(L0 + [1] * (3 - d)), lmax=lmax, r=r,
                          bc=oracle.BC_PERIODIC if periodic else oracle.BC_TRANSMISSIVE, auto_regrid=0)
    o = oracle.Oracle(cfg)
    o.set_initial(oracle.IC_CONST, [1.0, 0.0, 0.0, 0.0, 1.0][: o.V], nrefine=0)
    rng = np.random.default_rng(seed)
    for it in range(4 if d == 2 else 2):
        meta, _ = o.cells()
        p_ref = 0.08 if it < 2 else 0.03
        flags = np.where(rng.random(len(meta)) < p_ref, 1, 0).astype(np.int8)
        flags[(meta[:, 1] == -1) & (rng.random(len(meta)) < 0.5)] = -1
        o.regrid_with_flags(flags, init_mode=1)
        new_meta, _ = o.cells()
        check_tree(new_meta, lmax, L0, d, r, M, periodic, flags, meta)
        # zero flags: nothing changes
        o.regrid_with_flags(np.zeros(len(new_meta), dtype=np.int8), init_mode=1)
        again, _ = o.cells()
        assert np.array_equal(again, new_meta)


def test_coarsening_restores_uniform_grid():
    cfg = oracle.make_cfg(dim=2, M=2, n=(6, 6, 1), lmax=1, r=3, auto_regrid=0)
    o = oracle.Oracle(cfg)
    o.set_initial(oracle.IC_CONST, [1.0, 0.0, 0.0, 2.5], nrefine=0)
    meta0, _ = o.cells()
    flags = np.zeros(len(meta0), dtype=np.int8)
    flags[14] = 1
    o.regrid_with_flags(flags, init_mode=1)
    meta1, _ = o.cells()
    assert (meta1[:, 1] == -1).sum() == 1 and (meta1[:, 1] == 1).sum() == 8 * 9
    f = np.where(meta1[:, 1] == -1, -1, 0).astype(np.int8)
    o.regrid_with_flags(f, init_mode=1)
    meta2, _ = o.cells()
    assert np.array_equal(meta2, meta0)
