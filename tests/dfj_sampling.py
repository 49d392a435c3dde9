"""Sampled checks of DF-J outputs against the oracle: J blocks of random shell
pairs and gamma entries of random ket shells, each recomputed by the oracle
over exactly the triples the screened plan keeps (its exported task list)."""
import numpy as np

import oracle


def kept_kets(groups, a, b):
    """Every ket shell the screened plan keeps for the shell pair (a, b)."""
    out = []
    for gr in groups:
        hit = np.where((gr["pairs"][:, 0] == a) & (gr["pairs"][:, 1] == b))[0]
        for j in hit:
            out.extend(int(x) for x in gr["auxs"][:gr["counts"][j]])
    return out


def kept_pairs(groups, P):
    """Every shell pair the screened plan keeps for the ket shell P."""
    out = []
    for gr in groups:
        pos = np.where(gr["auxs"] == P)[0]
        if len(pos):
            out.extend(tuple(int(x) for x in ab) for ab in gr["pairs"][gr["counts"] > int(pos[0])])
    return out


ATOL = 1e-14  # the integral criterion's absolute term


def sampled_against_oracle(cl, plan, D, c, g, J, npair, nket, seed, mode, tol):
    """J blocks of npair random shell pairs and gamma of nket random ket
    shells against the oracle over exactly the triples the plan keeps.

    Each output is a dot product over many integrals I with weights w (c for
    J, w_ab D for gamma).  Integrals within tol |I| + ATOL of the oracle give
    an output within tol sum |I||w| + ATOL sum |w|: that bound, taken at the
    block's largest element, is the tolerance.  The ATOL term matters for
    blocks of pairs whose overlap is tiny (a compact shell and a far diffuse
    one), where every integral is far below 1e-14."""
    ao, aq = oracle.ao_offsets(cl.orb), oracle.ao_offsets(cl.aux)
    groups = plan.groups()
    rng = np.random.default_rng(seed)
    allpairs = np.concatenate([gr["pairs"] for gr in groups])
    for k in rng.choice(len(allpairs), size=npair, replace=False):
        a, b = (int(x) for x in allpairs[k])
        Ps = kept_kets(groups, a, b)
        blocks = oracle.eri3c_triples(cl.orb, cl.aux, [[a, b]] * len(Ps), Ps, mode=mode)
        ref = sum(np.einsum("abP,P->ab", X, c[aq[P]:aq[P + 1]]) for X, P in zip(blocks, Ps))
        # a J element is a dot product over the kept kets: its rounding scale is sum |I| |c|
        scale = sum(np.einsum("abP,P->ab", np.abs(X), np.abs(c[aq[P]:aq[P + 1]])) for X, P in zip(blocks, Ps))
        wsum = sum(np.abs(c[aq[P]:aq[P + 1]]).sum() for P in Ps)
        got = J[ao[a]:ao[a + 1], ao[b]:ao[b + 1]]
        err = np.abs(got - ref).max()
        assert err <= tol * scale.max() + ATOL * wsum, (a, b, err, scale.max(), wsum)
    for P in rng.choice(cl.aux.nshell, size=nket, replace=False):
        pairs = kept_pairs(groups, int(P))
        blocks = oracle.eri3c_triples(cl.orb, cl.aux, pairs, np.full(len(pairs), P), mode=mode)
        ref = np.zeros(2 * cl.aux.l[P] + 1)
        scale = np.zeros_like(ref)
        wsum = 0.0
        for (a, b), X in zip(pairs, blocks):
            w = 1.0 if a == b else 2.0
            Dab = D[ao[a]:ao[a + 1], ao[b]:ao[b + 1]]
            ref += w * np.einsum("abP,ab->P", X, Dab)
            scale += w * np.einsum("abP,ab->P", np.abs(X), np.abs(Dab))
            wsum += w * np.abs(Dab).sum()
        got = g[aq[P]:aq[P + 1]]
        err = np.abs(got - ref).max()
        assert err <= tol * scale.max() + ATOL * wsum, (P, err, scale.max(), wsum)
