"""Shared helpers of the GPU tests: engine construction from seeded inputs and
element-wise comparison with the oracle."""
import numpy as np

import oracle as orc
from paper_1006_4247_gb300 import pt
from paper_1006_4247_gb300 import workloads as W


def site_colour(L):
    x = np.arange(L ** 3)
    return ((x % L) + (x // L) % L + x // (L * L)) % 2


def make_engine(L, S=1, NT=4, C=2, precision="fp64", seed=11, jseed=100, bmin=0.5, bmax=2.0,
                start="random"):
    J = np.stack([W.couplings(L, jseed + s) for s in range(S)])
    B = np.stack([W.linear_betas(NT, bmin, bmax) for _ in range(S)])
    eng = pt.Engine(L, J, B, n_copies=C, precision=precision, seed=seed, start=start)
    return eng, J.astype(np.float64), B


def set_random_state(eng, S, C, NT, L, seed):
    """Put seeded random unit spins into every replica; return them as the
    engine stores them (rounded to the engine's precision)."""
    st = np.zeros((S, C, NT, L ** 3, 3))
    for s in range(S):
        for c in range(C):
            for b in range(NT):
                v = W.random_spins(L, seed + 1000 * s + 100 * c + b)
                eng.set_spins(s, c, b, v)
                st[s, c, b] = eng.get_spins(s, c, b)
    return st


def get_state(eng, S, C, NT):
    return np.stack([np.stack([np.stack([eng.get_spins(s, c, b) for b in range(NT)])
                               for c in range(C)]) for s in range(S)])


def ambiguous_basis_sites(L, J, s, colour, tol=1e-4):
    """Sites of `colour` whose neighbour field is nearly perpendicular to e_z:
    there the heat-bath basis of float and double arithmetic may pick
    opposite orientations (sign of S_z), so only the component along S and
    |s| = 1 are unique."""
    out = np.zeros(L ** 3, bool)
    col = site_colour(L)
    for x in np.nonzero(col == colour)[0]:
        S = orc.local_field(L, J, s, x)
        n = np.linalg.norm(S)
        out[x] = n == 0 or abs(S[2]) < tol * n
    return out


def u53(w0, w1):
    """The exchange uniform in [0, 1) from two Philox words: 53 bits, the
    upper 27 of w0 and 26 of w1."""
    return ((int(w0) >> 5) * 67108864 + (int(w1) >> 6)) * 2.0 ** -53


def metropolis(lnA, u):
    return lnA >= 0.0 or u < np.exp(lnA)


def exchange_walk(mode, L, J, betas, spins, H, seed, sample, copy, step, eps=None, follow_lnA=None):
    """One tempering update of one chain replayed pair by pair with the
    oracle's primitives (standard swap, Eq. 1; decimation, Eq. aswap with
    heat-bath re-insertion; cooling/heating, section III.B), so that the
    per-pair terms can be compared with the engine's exchange log.

    spins [NT][N][3] and H [NT] are the configurations and energies at each
    beta when the update starts (taken from the engine).  With follow_lnA
    (the engine's logged ln A of every pair) the walk takes the engine's
    decision, metropolis(follow_lnA[i], u), so that it stays on the engine's
    path where float round-off decides a pair; the oracle's own decision is
    kept beside it.  Returns a list of per-pair dicts (lnA, lnJ1, lnJ2, u,
    accepted, oracle_accepts, H1, H2) and the final spins, energies and
    permutation of the configurations."""
    NT = len(betas)
    sp = np.array(spins, dtype=np.float64, copy=True)
    H = np.array(H, dtype=np.float64, copy=True)
    perm = np.arange(NT)
    out = []
    d0 = int(orc.rng_words(seed, sample, 0, copy, step, 3)[0]) & 1
    for i in range(NT - 1):
        b1, b2 = float(betas[i]), float(betas[i + 1])
        w = orc.rng_words(seed, sample, i, copy, step, 1)
        u = u53(w[0], w[1])
        rec = {"lnJ1": 0.0, "lnJ2": 0.0, "u": u, "H1": H[i], "H2": H[i + 1]}
        if mode == "plain":
            lnA = (b2 - b1) * (H[i + 1] - H[i])
        elif mode == "decimation":
            d = (d0 + i) & 1
            lnA = orc.decimation_lnA(L, J, sp[i], sp[i + 1], d, b1, b2)
            rec["d"] = d
        else:
            e = float(eps[i])
            t1, lj1 = orc.cool_sweep(L, J, sp[i], e)
            t2, lj2 = orc.heat_sweep(L, J, sp[i + 1], e)
            Hc, Hh = orc.energy(L, J, t1), orc.energy(L, J, t2)
            lnA = -b2 * Hc - b1 * Hh + b1 * H[i] + b2 * H[i + 1] + lj1 - lj2
            rec.update(lnJ1=lj1, lnJ2=lj2, Hc=Hc, Hh=Hh)
        rec["lnA"] = lnA
        rec["oracle_accepts"] = metropolis(lnA, u)
        ok = rec["oracle_accepts"] if follow_lnA is None else metropolis(float(follow_lnA[i]), u)
        rec["accepted"] = ok
        if ok:
            perm[i], perm[i + 1] = perm[i + 1], perm[i]
            if mode == "plain":
                sp[[i, i + 1]] = sp[[i + 1, i]]
                H[i], H[i + 1] = H[i + 1], H[i]
            elif mode == "decimation":
                sp[[i, i + 1]] = sp[[i + 1, i]]
                rec["ambiguous"] = False
                for k, b in ((i, b1), (i + 1, b2)):
                    # float's S_z errs by ~1e-6 |S|: 1e-5 flags every site where the
                    # two precisions could take opposite signs
                    rec["ambiguous"] |= bool(ambiguous_basis_sites(L, J, sp[k], rec["d"], tol=1e-5).any())
                    sp[k] = orc.hb_halfsweep(L, J, sp[k], rec["d"], b, seed, sample, copy * NT + k, step,
                                             purpose=2)
                    H[k] = orc.energy(L, J, sp[k])
            else:
                sp[i], sp[i + 1] = t2, t1
                H[i], H[i + 1] = rec["Hh"], rec["Hc"]
        out.append(rec)
    return out, sp, H, perm


# Float exchanges against the oracle walk, element by element.  Bounds, from
# the arithmetic:
#   ln det J_f of one site is formed as log1p of a small argument from the
#   series values of cos(a) - 1 and sin(a)/a (relative error ~1e-7), so it
#   errs by a few 1e-8 plus what the site's inputs carry: the spins and the
#   field agree with the oracle's to ~1e-6, which moves eps S.s by at most
#   ~1e-6; LNJ_SITE = 1e-6 per site bounds it, N LNJ_SITE a sweep's sum.
#   Decimation: the per-site terms D(|S|) are O(1..10) values taken with the
#   accurate float log1p/exp, a few ulp each; with the fields' 1e-6 the two
#   terms of a site err by less than LNJ_SITE, N/2 sites by N LNJ_SITE.
#   Energies: a configuration's H is an exact fixed-point sum of per-site
#   float terms, so it errs by what the terms carry (the spins' ~1e-6, with
#   random signs over N sites); ENERGY_REL = 1e-7 of |H| bounds it with
#   margin.  Standard swap: (b2 - b1)(H2 - H1) with the engine's energies,
#   2e-5 relative (the energy tolerance of the parity tests).
# ln A must lie within its bound of the oracle walk's; where the two ln A
# lie on different sides of ln u the oracle's ln A must be within that bound
# of ln u (a round-off tie, after which the walk follows the engine).
# Transformed and re-inserted spins: 1e-5 per component (the float bound of
# one sweep).
LNJ_SITE = 1e-6
ENERGY_REL = 1e-7


def float_tolerances(recs, mode, betas, N):
    """Attach to every pair record of an oracle walk its ln A bound."""
    for i, r in enumerate(recs):
        b1, b2 = betas[i], betas[i + 1]
        if mode == "plain":
            r["tolA"] = (b2 - b1) * 2e-5 * (abs(r["H1"]) + abs(r["H2"]))
        elif mode == "decimation":
            r["tolA"] = N * LNJ_SITE
        else:
            hs = b1 * abs(r["H1"]) + b2 * abs(r["H2"]) + b2 * abs(r["Hc"]) + b1 * abs(r["Hh"])
            r["tolA"] = ENERGY_REL * hs + 2 * N * LNJ_SITE


def check_float_walk(errors, name, eng_lnA, eng_lnJ, recs, N):
    """Per pair: ln A and the Jacobian terms within their bounds, decisions
    equal outside the round-off band of ln u (largest errors and the number
    of ties kept in errors[name]).  Returns False if the walk met a
    re-insertion whose heat-bath basis float and double may orient oppositely
    (|S_z| < 1e-4 |S| at a site): the configurations part there, so the
    caller skips the final comparison of that chain."""
    errs = errors.setdefault(name, {"lnA": 0.0, "lnJ": 0.0, "spin": 0.0, "ties": 0, "pairs": 0})
    for i, r in enumerate(recs):
        dA = abs(eng_lnA[i] - r["lnA"])
        dJ = max(abs(eng_lnJ[i, 0] - r["lnJ1"]), abs(eng_lnJ[i, 1] - r["lnJ2"]))
        errs["lnA"] = max(errs["lnA"], float(dA))
        errs["lnJ"] = max(errs["lnJ"], float(dJ))
        errs["pairs"] += 1
        assert dJ <= N * LNJ_SITE, (name, i, dJ)
        assert dA <= r["tolA"], (name, i, dA, r["tolA"])
        if r["accepted"] != r["oracle_accepts"]:
            # accept iff ln u < ln A: a different decision needs ln u in the band
            assert abs(r["lnA"] - np.log(max(r["u"], 1e-300))) <= r["tolA"], (name, i)
            errs["ties"] += 1
        if r.get("ambiguous"):
            return False
    return True
