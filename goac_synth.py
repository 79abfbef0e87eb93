"""Seeded synthetic inputs shaped like the paper's workloads.

This module is the only code that both the CUDA path and the CPU oracle use.
It holds none of the method's arithmetic: it produces lattices (rows are the
lattice vectors, Angstrom), fractional coordinates, site classes, fixed
charges, species charges and counts, random populations and logits.  Energies,
potentials, Ewald sums and every optimiser step live on either side of it.

Workloads (sizes follow the paper's cells; structures the paper does not give
are replaced by synthetic stand-ins of the same shape):
  * ``rocksalt_problem(reps, a)``: rocksalt supercell, anions fixed at -2 and a
    cation class holding +1 / +3 in equal numbers (NaCl section of the paper).
  * ``layered_problem()``: R-3m layered-oxide-like 12x12x1 cell, N = 1296
    (the paper's 6x6x1 size of Table 1), Li/vacancy and 4-cation TM classes.
  * ``random_cubic_problem()``: jittered cubic grid, N = 4096, 4 species.
  * ``batch_problems()``: 256 rocksalt / spinel-like cells of uneven N.
  * ``bcc_relaxed_problem()``: bcc 16^3 cell, N = 8192, 5 species.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 0x600AC


@dataclass
class Problem:
    """A configurational problem: cell, sites, classes, species and counts."""
    name: str
    lattice: np.ndarray          # (3, 3) rows = lattice vectors (Angstrom)
    frac: np.ndarray             # (N, 3) fractional coordinates in [0, 1)
    site_class: np.ndarray       # (N,) int32, -1 fixed, else class index
    fixed_q: np.ndarray          # (N,) float64, charge of fixed sites (0 elsewhere)
    z: np.ndarray                # (S,) float64 species charges
    counts: np.ndarray           # (n_class, S) int32 species counts per class
    alpha: float                 # Ewald splitting parameter (1/Angstrom)
    nimg: tuple                  # real-space image box |n_a| <= nimg[a]
    kcut: float                  # reciprocal cutoff |k| <= kcut (1/Angstrom)
    species_names: list = field(default_factory=list)

    @property
    def N(self) -> int:
        return int(self.frac.shape[0])

    @property
    def Nv(self) -> int:
        return int((self.site_class >= 0).sum())

    @property
    def S(self) -> int:
        return int(self.z.shape[0])

    @property
    def n_class(self) -> int:
        return int(self.counts.shape[0])


def default_cutoffs(lattice: np.ndarray):
    """Cutoff recipe for a general cell: L = V^(1/3), alpha = 5/L,
    nimg_a = ceil((6/alpha) / width_a), kcut = 12 alpha (input parameters)."""
    A = np.asarray(lattice, dtype=np.float64)
    V = abs(float(np.linalg.det(A)))
    L = V ** (1.0 / 3.0)
    alpha = 5.0 / L
    nimg = []
    for a in range(3):
        b, c = A[(a + 1) % 3], A[(a + 2) % 3]
        width = V / float(np.linalg.norm(np.cross(b, c)))
        nimg.append(int(math.ceil((6.0 / alpha) / width)))
    return alpha, tuple(nimg), 12.0 * alpha


# --------------------------------------------------------------------------
# Crystal cells
# --------------------------------------------------------------------------
def _supercell(basis_frac, reps):
    """Tile fractional basis positions over reps = (na, nb, nc) cells."""
    na, nb, nc = reps
    out = []
    for i in range(na):
        for j in range(nb):
            for k in range(nc):
                for f in basis_frac:
                    out.append(((f[0] + i) / na, (f[1] + j) / nb, (f[2] + k) / nc))
    return np.array(out, dtype=np.float64) % 1.0


ROCKSALT_CATION = [(0, 0, 0), (0, .5, .5), (.5, 0, .5), (.5, .5, 0)]
ROCKSALT_ANION = [(.5, .5, .5), (.5, 0, 0), (0, .5, 0), (0, 0, .5)]


def rocksalt_cell(reps, a):
    """Conventional rocksalt supercell: (lattice, frac, is_anion)."""
    basis = ROCKSALT_CATION + ROCKSALT_ANION
    lab = [0] * 4 + [1] * 4
    frac = _supercell(basis, reps)
    # _supercell iterates cells outermost, basis innermost
    is_anion = np.tile(np.array(lab, dtype=bool), reps[0] * reps[1] * reps[2])
    lattice = np.diag([a * reps[0], a * reps[1], a * reps[2]]).astype(np.float64)
    return lattice, frac, is_anion


def cscl_cell(a):
    lattice = np.diag([a, a, a]).astype(np.float64)
    frac = np.array([[0, 0, 0], [.5, .5, .5]], dtype=np.float64)
    return lattice, frac, np.array([False, True])


def zincblende_cell(a):
    cat = [(0, 0, 0), (0, .5, .5), (.5, 0, .5), (.5, .5, 0)]
    an = [(.25, .25, .25), (.25, .75, .75), (.75, .25, .75), (.75, .75, .25)]
    lattice = np.diag([a, a, a]).astype(np.float64)
    return lattice, np.array(cat + an, dtype=np.float64), np.array([False] * 4 + [True] * 4)


# --------------------------------------------------------------------------
# Problems
# --------------------------------------------------------------------------
def rocksalt_problem(reps=(2, 2, 2), a=4.2, nimg=None, kcut_m=8):
    """Rocksalt supercell: anions fixed at -2; one cation class with +1 and +3
    in equal numbers.  alpha = 5/L, kcut = kcut_m * 2 pi / L, L = the longest
    edge; nimg defaults to 3 images along every axis."""
    lattice, frac, is_anion = rocksalt_cell(reps, a)
    N = frac.shape[0]
    site_class = np.where(is_anion, -1, 0).astype(np.int32)
    fixed_q = np.where(is_anion, -2.0, 0.0)
    ncat = int((~is_anion).sum())
    z = np.array([1.0, 3.0])
    counts = np.array([[ncat // 2, ncat - ncat // 2]], dtype=np.int32)
    L = float(max(lattice[0, 0], lattice[1, 1], lattice[2, 2]))
    return Problem(name=f"rocksalt{reps[0]}x{reps[1]}x{reps[2]}", lattice=lattice, frac=frac,
                   site_class=site_class, fixed_q=fixed_q, z=z, counts=counts,
                   alpha=5.0 / L, nimg=tuple(nimg) if nimg else (3, 3, 3),
                   kcut=kcut_m * 2.0 * math.pi / L, species_names=["M+1", "M+3"])


def layered_problem(reps=(12, 12, 1), a_h=2.88, c=14.2, z_o=0.25):
    """R-3m layered-oxide-like hexagonal supercell (alpha-NaFeO2 type).

    Per hexagonal cell: TM on 3a, Li layer on 3b and the +z member of each O 6c
    pair (3 O), so 9 sites per cell and N = 1296 for 12x12x1.  Li layer: Li+
    346 and vacancies 86; TM layer: Ni2+, Ni3+, Mn4+, Co3+ 108 each; every O
    carries the neutralising charge -(346 + 1296)/432."""
    shifts = [(0.0, 0.0, 0.0), (2 / 3, 1 / 3, 1 / 3), (1 / 3, 2 / 3, 2 / 3)]
    tm = [s for s in shifts]
    li = [(s[0], s[1], (s[2] + 0.5) % 1.0) for s in shifts]
    ox = [(s[0], s[1], (s[2] + z_o) % 1.0) for s in shifts]
    basis = tm + li + ox
    lab = [1] * 3 + [0] * 3 + [-1] * 3
    frac = _supercell(basis, reps)
    ncell = reps[0] * reps[1] * reps[2]
    site_class = np.tile(np.array(lab, dtype=np.int32), ncell)
    n_o = int((site_class == -1).sum())
    n_li_sites = int((site_class == 0).sum())
    n_tm = int((site_class == 1).sum())
    n_li = int(math.floor(0.8 * n_li_sites + 0.5))
    z = np.array([1.0, 0.0, 2.0, 3.0, 4.0, 3.0])
    names = ["Li+", "Vac", "Ni2+", "Ni3+", "Mn4+", "Co3+"]
    q_tm = n_tm // 4
    counts = np.zeros((2, 6), dtype=np.int32)
    counts[0, 0], counts[0, 1] = n_li, n_li_sites - n_li
    counts[1, 2:6] = [q_tm, q_tm, q_tm, n_tm - 3 * q_tm]
    cation_charge = float(counts[0] @ z + counts[1] @ z)
    q_o = -cation_charge / n_o
    fixed_q = np.where(site_class == -1, q_o, 0.0)
    a1 = np.array([a_h * reps[0], 0.0, 0.0])
    a2 = np.array([-0.5 * a_h * reps[1], math.sqrt(3) / 2 * a_h * reps[1], 0.0])
    a3 = np.array([0.0, 0.0, c * reps[2]])
    lattice = np.stack([a1, a2, a3])
    alpha, nimg, kcut = default_cutoffs(lattice)
    return Problem(name=f"layered{reps[0]}x{reps[1]}x{reps[2]}", lattice=lattice, frac=frac, site_class=site_class, fixed_q=fixed_q,
                   z=z, counts=counts, alpha=alpha, nimg=nimg, kcut=kcut, species_names=names)


def random_cubic_problem(n_side=16, spacing=2.5, jitter=0.3, seed=SEED_BASE + 2):
    """Jittered simple-cubic grid (N = n_side^3), one class holding +1, +2, +3
    and -2 in counts N/8, N/4, N/8, N/2 (neutral)."""
    rng = np.random.default_rng(seed)
    L = n_side * spacing
    g = np.arange(n_side, dtype=np.float64)
    gx, gy, gz = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1) * spacing
    pos = pos + rng.uniform(-jitter, jitter, size=pos.shape)
    frac = (pos / L) % 1.0
    N = frac.shape[0]
    site_class = np.zeros(N, dtype=np.int32)
    z = np.array([1.0, 2.0, 3.0, -2.0])
    counts = np.array([[N // 8, N // 4, N // 8, N // 2]], dtype=np.int32)
    lattice = np.diag([L, L, L]).astype(np.float64)
    alpha, nimg, kcut = default_cutoffs(lattice)
    return Problem(name=f"randcubic{N}", lattice=lattice, frac=frac, site_class=site_class,
                   fixed_q=np.zeros(N), z=z, counts=counts, alpha=alpha, nimg=nimg, kcut=kcut,
                   species_names=["+1", "+2", "+3", "-2"])


def bcc_relaxed_problem(n_side=16, a=3.0):
    """bcc (CsCl positions) n_side^3 conventional cells, all 2 n_side^3 sites in
    one class with 5 species (+1, +2, +3, +4, 0) in near-equal counts."""
    frac = _supercell([(0, 0, 0), (.5, .5, .5)], (n_side, n_side, n_side))
    N = frac.shape[0]
    z = np.array([1.0, 2.0, 3.0, 4.0, 0.0])
    base = N // 5
    cnt = [base] * 5
    for r in range(N - 5 * base):
        cnt[r] += 1
    lattice = np.diag([a * n_side] * 3).astype(np.float64)
    alpha, nimg, kcut = default_cutoffs(lattice)
    return Problem(name=f"bcc{N}", lattice=lattice, frac=frac, site_class=np.zeros(N, dtype=np.int32),
                   fixed_q=np.zeros(N), z=z, counts=np.array([cnt], dtype=np.int32), alpha=alpha, nimg=nimg,
                   kcut=kcut, species_names=["+1", "+2", "+3", "+4", "0"])


SPINEL_A = [(1 / 8, 1 / 8, 1 / 8), (7 / 8, 3 / 8, 3 / 8)]          # 8a (origin choice 2), 2 of the fcc-centred set
SPINEL_B = [(1 / 2, 1 / 2, 1 / 2), (1 / 2, 1 / 4, 1 / 4), (1 / 4, 1 / 2, 1 / 4), (1 / 4, 1 / 4, 1 / 2)]  # 16d


def _spinel_cell():
    """Spinel-like cubic cell (Fd-3m, origin choice 2): 8 A + 16 B cations and
    32 O at x = 0.26, fcc translations applied."""
    fcc = [(0, 0, 0), (0, .5, .5), (.5, 0, .5), (.5, .5, 0)]
    x = 0.26
    o_base = [(x, x, x), (-x + 0.5, -x + 0.5, x), (x, -x + 0.5, -x + 0.5), (-x + 0.5, x, -x + 0.5),
              (-x + 0.25, -x + 0.25, -x + 0.25), (x + 0.75, x + 0.75, -x + 0.25),
              (-x + 0.25, x + 0.75, x + 0.75), (x + 0.75, -x + 0.25, x + 0.75)]

    def expand(b):
        out = []
        for f in fcc:
            for p in b:
                out.append(tuple((p[d] + f[d]) % 1.0 for d in range(3)))
        return out
    return expand(SPINEL_A), expand(SPINEL_B), expand(o_base)


def batch_problems(n_cells=256, seed=SEED_BASE + 3, n_min=64, n_max=2048):
    """Uneven batch of rocksalt / spinel-like cells.  Each cell: N drawn
    log-uniformly in [n_min, n_max] and mapped to the nearest supercell; 2..5
    cation species with charges in +1..+4 (repeats allowed) on one cation class;
    anions fixed at -2; counts from a Dirichlet(1) draw rounded and then
    adjusted one at a time towards neutrality; kT ~ U(0.01, 0.2) eV."""
    rng = np.random.default_rng(seed)
    a_sp, b_sp, o_sp = _spinel_cell()
    out = []
    for _ in range(n_cells):
        target = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        kind = "rocksalt" if rng.uniform() < 0.5 else "spinel"
        per = 8 if kind == "rocksalt" else 56
        best = None
        for na in range(1, 9):
            for nb in range(na, 9):
                for nc in range(nb, 9):
                    n = per * na * nb * nc
                    if n > n_max * 1.2:
                        continue
                    score = abs(math.log(n / target))
                    if best is None or score < best[0]:
                        best = (score, (na, nb, nc))
        reps = best[1]
        if kind == "rocksalt":
            lattice, frac, is_anion = rocksalt_cell(reps, 4.2)
        else:
            basis = a_sp + b_sp + o_sp
            lab = [False] * (len(a_sp) + len(b_sp)) + [True] * len(o_sp)
            frac = _supercell(basis, reps)
            is_anion = np.tile(np.array(lab), reps[0] * reps[1] * reps[2])
            lattice = np.diag([8.1 * reps[0], 8.1 * reps[1], 8.1 * reps[2]]).astype(np.float64)
        n_an = int(is_anion.sum())
        n_cat = int((~is_anion).sum())
        target_charge = 2 * n_an
        for _attempt in range(200):
            k = int(rng.integers(2, 6))
            z = rng.integers(1, 5, size=k).astype(np.float64)
            w = rng.dirichlet(np.ones(k))
            cnt = np.floor(w * n_cat).astype(np.int64)
            while cnt.sum() < n_cat:
                cnt[int(rng.integers(0, k))] += 1
            ok = False
            for _step in range(4 * n_cat):
                charge = float(cnt @ z)
                if charge == target_charge:
                    ok = True
                    break
                if charge < target_charge:
                    lo = [s for s in range(k) if cnt[s] > 0]
                    hi = [s for s in range(k) if z[s] > min(z[t] for t in lo)]
                    if not hi:
                        break
                    s_from = min(lo, key=lambda s: z[s])
                    s_to = max(range(k), key=lambda s: z[s])
                else:
                    lo = [s for s in range(k) if cnt[s] > 0]
                    s_from = max(lo, key=lambda s: z[s])
                    s_to = min(range(k), key=lambda s: z[s])
                if z[s_to] == z[s_from]:
                    break
                cnt[s_from] -= 1
                cnt[s_to] += 1
            if ok and (cnt > 0).sum() >= 2 and len(set(z[cnt > 0].tolist())) >= 2:
                break
        site_class = np.where(is_anion, -1, 0).astype(np.int32)
        fixed_q = np.where(is_anion, -2.0, 0.0)
        alpha, nimg, kcut = default_cutoffs(lattice)
        prob = Problem(name=f"{kind}{reps}", lattice=lattice, frac=frac, site_class=site_class, fixed_q=fixed_q,
                       z=z, counts=cnt.reshape(1, -1).astype(np.int32), alpha=alpha, nimg=nimg, kcut=kcut)
        prob.kT = float(rng.uniform(0.01, 0.2))
        out.append(prob)
    return out


# --------------------------------------------------------------------------
# Populations and other random inputs
# --------------------------------------------------------------------------
def random_population(prob: Problem, B: int, seed: int) -> np.ndarray:
    """B uniformly random count-preserving configurations (B x Nv int8)."""
    rng = np.random.default_rng(seed)
    nv = prob.Nv
    out = np.empty((B, nv), dtype=np.int8)
    vclass = prob.site_class[prob.site_class >= 0]
    for k in range(prob.n_class):
        idx = np.nonzero(vclass == k)[0]
        base = np.repeat(np.arange(prob.S, dtype=np.int8), prob.counts[k])
        assert base.shape[0] == idx.shape[0], "counts do not fill the class"
        for b in range(B):
            out[b, idx] = rng.permutation(base)
    return out


def random_logits(prob: Problem, B: int, seed: int, dtype=np.float32) -> np.ndarray:
    """Logits ~ N(0, 1) per (config, variable site, species): B x Nv x S."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((B, prob.Nv, prob.S)).astype(dtype)


def tiny_rocksalt_problem():
    """1x1x2 rocksalt cell: 8 anions fixed at -2 and 8 cations 4 x +1 / 4 x +3
    (70 configurations), the brute-force cell."""
    return rocksalt_problem(reps=(1, 1, 2), a=4.2)


def o3_layered_problem(reps=(2, 2, 1), a_sqrt3=5.0, c=19.2, z_o=0.25):
    """O3 layered oxide of the paper's scaling study (Section "High-Entropy
    Layered Oxides", Table 1): Na2/3[Li1/6 Fe1/6 Co1/6 Ni1/6 Mn1/3]O2 in a
    sqrt(3) cell (a = 5.0 A, c = 19.2 A) with 9 Na positions (6 Na + 3
    vacancies), 9 TM positions (Li 1.5, Fe 1.5, Co 1.5, Ni 1.5, Mn 3) and 18 O
    per cell; charges Na+ Li+ Fe2.5+ Co3.5+ Ni2+ Mn4+ O1.75-.  Positions: the
    alpha-NaFeO2 (R-3m) arrangement of a hexagonal cell with a_h = a/sqrt(3)
    (TM 3a, Na 3b, O 6c at z = +-z_o; the paper does not give z), re-expressed in
    the sqrt(3) x sqrt(3) cell and tiled reps times."""
    ah = a_sqrt3 / math.sqrt(3.0)
    h1 = np.array([ah, 0.0, 0.0])
    h2 = np.array([-0.5 * ah, math.sqrt(3) / 2 * ah, 0.0])
    h3 = np.array([0.0, 0.0, c])
    b1, b2 = h1 - h2, h1 + 2 * h2
    cell = np.stack([b1, b2, h3])
    rshift = [(0.0, 0.0, 0.0), (2 / 3, 1 / 3, 1 / 3), (1 / 3, 2 / 3, 2 / 3)]
    basis = []
    for s in rshift:
        basis.append(((s[0], s[1], s[2] % 1.0), 1))              # TM 3a
        basis.append(((s[0], s[1], (s[2] + 0.5) % 1.0), 0))      # Na 3b
        basis.append(((s[0], s[1], (s[2] + z_o) % 1.0), -1))     # O 6c
        basis.append(((s[0], s[1], (s[2] - z_o) % 1.0), -1))
    inv = np.linalg.inv(cell)
    pts, labs = [], []
    for i in range(-3, 4):
        for j in range(-3, 4):
            for f, lab in basis:
                r = (f[0] + i) * h1 + (f[1] + j) * h2 + f[2] * h3
                g = r @ inv
                g = np.where(np.abs(g - np.round(g)) < 1e-9, np.round(g), g)
                if np.all(g >= -1e-9) and np.all(g < 1 - 1e-9):
                    pts.append(g % 1.0)
                    labs.append(lab)
    pts = np.array(pts)
    labs = np.array(labs)
    order = np.lexsort((pts[:, 0], pts[:, 1], pts[:, 2], labs))
    pts, labs = pts[order], labs[order]
    assert (labs == 0).sum() == 9 and (labs == 1).sum() == 9 and (labs == -1).sum() == 18
    frac = _supercell([tuple(p) for p in pts], reps)
    ncell = reps[0] * reps[1] * reps[2]
    site_class = np.tile(labs.astype(np.int32), ncell)
    z = np.array([1.0, 0.0, 1.0, 2.5, 3.5, 2.0, 4.0])
    names = ["Na+", "Vac", "Li+", "Fe2.5+", "Co3.5+", "Ni2+", "Mn4+"]
    counts = np.zeros((2, 7), dtype=np.int32)
    counts[0, 0], counts[0, 1] = 6 * ncell, 3 * ncell
    h = (3 * ncell) // 2
    counts[1, 2:7] = [h, h, h, h, 3 * ncell]
    assert counts[1].sum() == 9 * ncell, "the TM counts need an even number of sqrt(3) cells"
    fixed_q = np.where(site_class == -1, -1.75, 0.0)
    lattice = cell * np.array(reps, dtype=np.float64)[:, None]
    alpha, nimg, kcut = default_cutoffs(lattice)
    return Problem(name=f"O3_{reps[0]}x{reps[1]}x{reps[2]}", lattice=lattice, frac=frac, site_class=site_class,
                   fixed_q=fixed_q, z=z, counts=counts, alpha=alpha, nimg=nimg, kcut=kcut, species_names=names)


#: the eight sqrt(3)-supercells of Table 1
TABLE1_CELLS = [(2, 2, 1), (2, 2, 2), (4, 4, 1), (4, 4, 2), (6, 6, 1), (8, 8, 1), (6, 6, 2), (6, 6, 3)]


def nacl_problem(reps=(3, 3, 3), a=5.62):
    """NaCl supercell of the paper's rocksalt study (Section "Atomistic
    Configurations in NaCl"): every position of the rocksalt lattice in one
    class, half Na+ and half Cl- (216 positions, 108 / 108 for 3x3x3, about
    10^64 configurations); the known optimum is rocksalt order, which is
    returned as `is_anion` (species 1 = Cl- on the anion sublattice)."""
    lattice, frac, is_anion = rocksalt_cell(reps, a)
    n = frac.shape[0]
    L = float(np.cbrt(abs(np.linalg.det(lattice))))
    prob = Problem(name=f"NaCl{reps[0]}x{reps[1]}x{reps[2]}", lattice=lattice, frac=frac,
                   site_class=np.zeros(n, np.int32), fixed_q=np.zeros(n), z=np.array([1.0, -1.0]),
                   counts=np.array([[n // 2, n // 2]], np.int32), alpha=5.0 / L, nimg=(2, 2, 2),
                   kcut=8 * 2 * math.pi / L, species_names=["Na+", "Cl-"])
    return prob, np.asarray(is_anion, dtype=np.int8)
