"""Test helpers built on the FP64 oracle alone (no CUDA path): which queries
have a ReLU mask that a binary32 evaluation may decide either way, and a
training batch in which such queries carry no gradient."""
import numpy as np

from oracle import octaoctree_oracle as O
from paper_2606_08469_gb300 import inputs as I

# a bound on the FP32 forward's error in a hidden pre-activation relative to
# sum |w||a| (256 units in the last place: the inputs' own rounding plus a
# 64-term dot product, per layer, with room to spare)
FP32_AMBIGUITY = 2.0 ** -16


def ambiguous_queries(ot, tables, weights, X, Om, gamma=FP32_AMBIGUITY):
    """Queries whose FP64 forward has a hidden pre-activation z with
    |z| <= gamma sum|w||a| (its ReLU mask may be taken either way in FP32),
    and the FP64 radiance of every query."""
    T = np.asarray(tables, np.float64)
    _, h, _, _ = O._encode(ot, T, X, Om, "cell")
    rgb, zs, inputs = O.mlp_forward(weights, h)
    amb = np.zeros(len(X), bool)
    for i, z in enumerate(zs[:-1]):
        W = np.asarray(weights[i], np.float64)
        amb |= np.any(np.abs(z) <= gamma * (np.abs(inputs[i]) @ np.abs(W).T), axis=1)
    return amb, rgb


def unambiguous_pairs(ot, tables, weights, pairs):
    """The pairs with every pair that has an ambiguous primary or secondary
    query given a zero residual: E = its FP64 primary radiance (rounded to
    FP32) and w = 0, so neither of its queries carries a gradient."""
    n = pairs.n
    X = np.concatenate([pairs.x, pairs.x2])
    Om = np.concatenate([pairs.omega, -pairs.omega2])
    amb, rgb = ambiguous_queries(ot, tables, weights, X, Om)
    bad = amb[:n] | amb[n:]
    E, w = pairs.E.copy(), pairs.w.copy()
    E[bad] = rgb[:n][bad].astype(np.float32)
    w[bad] = 0.0
    return I.TrainingPairs(pairs.x, pairs.omega, pairs.x2, pairs.omega2, E, w), \
        int(bad.sum())


def decoder_ambiguous(weights, h, gamma=FP32_AMBIGUITY):
    """Rows of the decoder input h whose FP64 forward has a hidden
    pre-activation within gamma sum|w||a| of zero."""
    _, zs, inputs = O.mlp_forward(weights, h)
    amb = np.zeros(len(h), bool)
    for i, z in enumerate(zs[:-1]):
        W = np.asarray(weights[i], np.float64)
        amb |= np.any(np.abs(z) <= gamma * (np.abs(inputs[i]) @ np.abs(W).T), axis=1)
    return amb


def predictor_ambiguous(table, res, pweights, X, Om, Nr, gamma=FP32_AMBIGUITY):
    """Queries whose g_psi forward (FP64) has an ambiguous hidden ReLU mask."""
    inp = np.concatenate([O.hash_encode(table, res, X), O.reflect_f32(Om, Nr).astype(np.float64)],
                         axis=1)
    return decoder_ambiguous(pweights, inp, gamma)


def lookup_unstable(ot, tables, X, Om, Nr, d32, rel=2.0 ** -16):
    """Queries whose shifted lookup decides another cell triangle or vertex
    when d moves by a relative rel either way (their binary32 decisions may
    differ between two FP32 evaluations of d)."""
    d32 = np.asarray(d32, np.float32)
    a0 = O.encode_features_shifted(ot, tables, X, Om, Nr, d32).addr
    bad = np.zeros(len(X), bool)
    for s in (1.0 + rel, 1.0 - rel):
        a = O.encode_features_shifted(ot, tables, X, Om, Nr, (d32 * np.float32(s)).astype(np.float32)).addr
        bad |= np.any(a != a0, axis=(1, 2, 3))
    return bad


def neutralise_pairs(pairs, bad, Lp):
    """The pairs with pair i given a zero residual where bad[i]: E = Lp[i]
    (its FP64 primary radiance rounded to FP32) and w = 0, so neither of its
    queries carries a gradient."""
    E, w = pairs.E.copy(), pairs.w.copy()
    E[bad] = Lp[bad].astype(np.float32)
    w[bad] = 0.0
    return I.TrainingPairs(pairs.x, pairs.omega, pairs.x2, pairs.omega2, E, w)
