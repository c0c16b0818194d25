"""Pins of the oracle's Eq. (2) step against an independent restatement (no GPU).

The reference below is written from the general multi-phase form of Eq. (2) (Sec. 2): for the
n phases present at a vertex (the layers of its closed neighbourhood and the base),

    dphi_i/dt = - sum_j (mu_ij / n) ( sum_k [ (w_ik - w_jk) phi_k + 1/2 (a_ik^2 - a_jk^2) lap phi_k ]
                                      - e_ij sqrt(phi_i phi_j) ),

with full n x n coefficient matrices: w_ij = a/5 and a_ij = 1/25 off the diagonal, 0 on it; mu_ij and
e_ij non-zero only between a layer and the base (Sec. 2, "Implementation details"), e antisymmetric
(+e for (layer, base): the front grows into the base).  Then one explicit Euler step, clamp to
[0, 1], snap at eps0 and 1 - eps0, and division by the column sum.  Nothing here shares code with
the oracle's per-vertex routine: the oracle applies a reduced two-term formula per layer, this
applies the matrix form, so a wrong mu/n (n = 2 at a three-phase vertex), a flipped sign of e or of
the w term, or a dropped Laplacian term shows as a mismatch.

  * step 1 on the torus and a genus-2 chain: every updated value against its hand-expanded 1-ring
    closed form (the seed's closed 1-ring at 1, everything else base);
  * the step of the first merge (torus, genus-2 chain): every frontier row, including the rows where
    two fronts and the base meet (n = 3), against the reference; the merged value at a collision
    row is the sum of its layers' new values (Sec. 3.1);
  * the same comparison with the reference's n replaced by 2 at the three-phase rows must fail:
    the check is sensitive to the branch it pins.
"""
import math

import numpy as np
import pytest

import meshgen
import oracle

ALIVE, DEAD, ENDED = 1, 2, 4


def consts():
    c = oracle.constants()
    a = 1.0 / 25.0
    return dict(mu=0.25, e=1.0 / 30.0, a=a, w=a / 5.0, dt=c["dt"], s=c["s"], eps0=1e-3)


def adjacency(m):
    nbr = [set() for _ in range(m.nv)]
    for f in m.F:
        for k in range(3):
            a, b = int(f[k]), int(f[(k + 1) % 3])
            nbr[a].add(b)
            nbr[b].add(a)
    return [sorted(x) for x in nbr]


def eq2_step(vals, laps, base, C, n_override=None):
    """One Euler step of the matrix form of Eq. (2) at one vertex.  vals / laps: the phases' values
    and Laplacians (index `base` is the base).  Returns the normalised new values."""
    n = len(vals)
    nn = n if n_override is None else n_override
    off = 1.0 - np.eye(n)
    W, A = C["w"] * off, C["a"] * off
    MU = np.zeros((n, n))
    E = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if (i == base) != (j == base):
                MU[i, j] = C["mu"]
                E[i, j] = C["e"] if j == base else -C["e"]
    x, L = np.asarray(vals, float), np.asarray(laps, float)
    rate = np.zeros(n)
    for i in range(n):
        for j in range(n):
            inner = sum((W[i, k] - W[j, k]) * x[k] + 0.5 * (A[i, k] ** 2 - A[j, k] ** 2) * L[k] for k in range(n))
            rate[i] -= MU[i, j] / nn * (inner - E[i, j] * math.sqrt(max(x[i] * x[j], 0.0)))
    y = np.clip(x + C["dt"] * rate, 0.0, 1.0)
    y[y < C["eps0"]] = 0.0
    y[y > 1.0 - C["eps0"]] = 1.0
    return y / y.sum()


def reference_step(m, nbr, layer, phi, lstate, C, n3_override=None):
    """New per-vertex total of the non-base layers after one step from the state (layer, phi)
    (one layer per vertex at a step boundary), and the rows where n = 3 phases met.  Frontier rows:
    not frozen, with the base and a live layer in the closed neighbourhood; a frozen plateau (a dead
    or ended layer) is read as the row's own layer at value 1 (a plateau is always enclosed by
    descendants of its layer)."""
    s = C["s"]

    def frozen(u):
        return layer[u] > 0 and lstate[layer[u]] in (DEAD, ENDED)

    out = phi.copy()
    rows3 = []
    for v in range(m.nv):
        if frozen(v):
            continue
        ring = [v] + nbr[v]
        layers, has_base = set(), False
        for u in ring:
            if frozen(u):
                continue
            if layer[u] > 0 and lstate[layer[u]] == ALIVE:
                layers.add(int(layer[u]))
            if 1.0 - (phi[u] if layer[u] > 0 else 0.0) > 0.0:
                has_base = True
        if not (has_base and layers):
            continue
        own = int(layer[v]) if layer[v] > 0 and lstate[layer[v]] == ALIVE else 0
        ls = sorted(layers)

        def val(u, l):
            if frozen(u):
                return 1.0 if (own != 0 and l == own) else 0.0
            return float(phi[u]) if layer[u] == l else 0.0

        def base(u):
            return 1.0 - (float(phi[u]) if layer[u] > 0 else 0.0)

        d = len(nbr[v])
        vals = [val(v, l) for l in ls] + [base(v)]
        laps = [s / d * sum(val(u, l) for u in nbr[v]) - s * val(v, l) for l in ls]
        laps.append(s / d * sum(base(u) for u in nbr[v]) - s * base(v))
        n_over = n3_override if (n3_override is not None and len(ls) == 2) else None
        y = eq2_step(vals, laps, len(ls), C, n_over)
        if len(ls) >= 2 and (y[:-1] > 0).sum() >= 2:
            rows3.append(v)
        out[v] = float(y[:-1].sum())
    return out, rows3


@pytest.mark.parametrize("which", ["torus", "chain2"])
def test_step_one_against_hand_expanded_ring(which):
    """After step 1 from the seed's closed 1-ring at value 1: a ring vertex with k of its d
    neighbours at 1 has Laplacians -s (d - k)/d (layer) and +s (d - k)/d (base), so Eq. (2) with n = 2
    gives rate (mu/2)(w - a^2 s (d-k)/d); a vertex outside the ring with k ring neighbours has rate
    (mu/2)(a^2 s k/d - w) (the sqrt term vanishes on both).  Euler, clamp, snap, normalise."""
    m = meshgen.torus(64, 32, 2.0, 0.7) if which == "torus" else meshgen.tube_chain(2, 64)
    seed = meshgen.seed_vertex(0, m.nv)
    C = consts()
    nbr = adjacency(m)
    ring = {seed, *nbr[seed]}
    r = oracle.detect(m, seed, max_steps=1, tunnels=0)
    mu, a, w, s, dt, eps0 = C["mu"], C["a"], C["w"], C["s"], C["dt"], C["eps0"]
    checked = 0
    for v in range(m.nv):
        d = len(nbr[v])
        k = sum(u in ring for u in nbr[v])
        if v in ring:
            if k == d:
                expect = 1.0  # no base in the closed neighbourhood: not updated
            else:
                y = 1.0 + dt * (mu / 2) * (w - a * a * s * (d - k) / d)
                yb = 0.0 - dt * (mu / 2) * (w - a * a * s * (d - k) / d)
                y, yb = min(max(y, 0.0), 1.0), min(max(yb, 0.0), 1.0)
                y = 0.0 if y < eps0 else (1.0 if y > 1 - eps0 else y)
                yb = 0.0 if yb < eps0 else (1.0 if yb > 1 - eps0 else yb)
                expect = y / (y + yb)
        elif k > 0:
            rate = (mu / 2) * (a * a * s * k / d - w)
            y, yb = min(max(dt * rate, 0.0), 1.0), min(max(1.0 - dt * rate, 0.0), 1.0)
            y = 0.0 if y < eps0 else (1.0 if y > 1 - eps0 else y)
            yb = 0.0 if yb < eps0 else (1.0 if yb > 1 - eps0 else yb)
            expect = y / (y + yb)
        else:
            expect = 0.0
        assert abs(r.phi[v] - expect) <= 1e-14, (v, d, k, r.phi[v], expect)
        checked += v in ring or k > 0
    assert checked > len(ring)


@pytest.mark.parametrize("which", ["torus", "chain2"])
def test_merge_step_against_matrix_form(which):
    m = meshgen.torus(64, 32, 2.0, 0.7) if which == "torus" else meshgen.tube_chain(2, 64)
    seed = meshgen.seed_vertex(0, m.nv)
    full = oracle.detect(m, seed, tunnels=0)
    t = next(st for kind, st in full.events() if kind == "MERGE")
    before = oracle.detect(m, seed, max_steps=t - 1, tunnels=0)
    after = oracle.detect(m, seed, max_steps=t, tunnels=0)
    lstate = {l + 1: int(before.layers[l, 2]) for l in range(len(before.layers))}
    assert (before.layer >= 0).all()  # one layer per vertex at a step boundary
    C = consts()
    nbr = adjacency(m)
    ref, rows3 = reference_step(m, nbr, before.layer, before.phi, lstate, C)
    assert len(rows3) > 0, "no three-phase collision row at the merge step"
    err = np.abs(ref - after.phi)
    assert err.max() <= 1e-14, f"max |reference - oracle| = {err.max():.3e} at vertex {int(err.argmax())}"
    # the merged value at a collision row is the sum of its layers' new values (one merged layer)
    assert all(after.layer[v] > 0 for v in rows3)
    # sensitivity: mu / 2 instead of mu / 3 at the three-phase rows is detected
    wrong, _ = reference_step(m, nbr, before.layer, before.phi, lstate, C, n3_override=2)
    assert np.abs(wrong - after.phi)[rows3].max() > 1e-6
