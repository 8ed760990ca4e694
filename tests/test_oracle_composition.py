"""Pins of the oracle's frame loop (Alg. 1 main thread + Alg. 2 assistant
threads): the order in which a frame takes s_c, the keystream slices of its
rounds and the two phases of each round.  These facts are fixed nowhere else:
the round trip cannot see them, because decryption mirrors whatever slicing
encryption uses.

The expected frames are rebuilt here, in numpy, from parts pinned on their own
(test_oracle_pins.py) and from the algorithm's statement:

* Alg. 1: PRBG_m keyed by K gives the subframe parameters P_m (four 6-byte
  groups per PLCM or logistic subframe, six per 2DLASM subframe), then one
  group per frame for s_c = 1 + (U mod 65536);
* Alg. 2 / Sec. 3: subframe i's PRBG is one continuous byte stream from x_1 on;
  frame f takes the next r S_i bytes and round j of it uses bytes
  [j S_i, (j + 1) S_i) of those;
* each round is the whole-frame confusion (Eq. 1) followed by the
  per-subframe diffusion (Eq. 3) seeded by the last byte of subframe
  (i + 1) mod n of the confused frame; decryption runs Eq. 4 then Eq. 2 with
  rounds r - 1 .. 0.

In the first test every number comes from exact integer arithmetic: PRBG_m
and every PRBG_a^i run the PLCM at p = 1/4 on dyadic starting values, where
Eq. 5 is exactly x -> 4x or 4x - 1 after the reflection.  The mutation test
shows that each plausible slip in the composition (round slices reversed or
cut per frame, diffusion before confusion, the next frame's s_c, the seed
taken after diffusion) changes the ciphertext, so these tests would catch it.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import synth
from tests.test_oracle_pins import _bits_of_dyadic, _plcm_int_orbit

mpmath = pytest.importorskip("mpmath")

_M48 = (1 << 48) - 1


# --------------------------------------------------------------- exact streams

def _exact_pair_stream(X1: int, X2: int, nbytes: int) -> np.ndarray:
    """Sec. 3 byte stream of a PLCM pair at p = 1/4 from x0 = X/2^52: the
    mantissa bytes (low 48 bits, LSB first) of the exact orbits, XORed."""
    steps = (nbytes + 5) // 6
    o1, o2 = _plcm_int_orbit(X1, steps), _plcm_int_orbit(X2, steps)
    out = bytearray()
    for a, b in zip(o1, o2):
        out += ((_bits_of_dyadic(a) ^ _bits_of_dyadic(b)) & _M48).to_bytes(6, "little")
    return np.frombuffer(bytes(out[:nbytes]), dtype=np.uint8)


def _groups(stream: np.ndarray) -> list[int]:
    """Consecutive 6-byte groups U (LSB first) of a PRBG_m stream."""
    return [int.from_bytes(stream[6 * g: 6 * g + 6].tobytes(), "little") for g in range(len(stream) // 6)]


def _unit(U: int) -> float:
    """u = (U + 1/2) 2^-48, exact in binary64."""
    return float(Fraction(2 * U + 1, 1 << 49))


# --------------------------------------------------------------- the composition

def _bounds(H, W, C, n):
    P = H * W
    return [C * ((i * P) // n) for i in range(n + 1)]


def _ktable(H: int, sc: int, orc) -> np.ndarray:
    """Eq. 1's k(alpha) = floor(s_c sin(2 pi alpha / H)): the oracle's table,
    itself checked here against the exact sine away from integers."""
    k = orc.ktable(H, sc)
    mpmath.mp.prec = 120
    for a in range(H):
        v = sc * mpmath.sin(2 * mpmath.pi * a / H)
        if abs(v - mpmath.nint(v)) > 1e-9:
            assert k[a] == int(mpmath.floor(v))
    return k


def _perm(H: int, W: int, k: np.ndarray):
    """Eq. 1 as index arrays: pixel (a, o) moves to (alpha, beta)."""
    a, o = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    alpha = (a + o) % H
    beta = (o + k[alpha]) % W
    return alpha, beta


def _confuse(X: np.ndarray, k: np.ndarray) -> np.ndarray:
    H, W, _ = X.shape
    alpha, beta = _perm(H, W, k)
    Y = np.empty_like(X)
    Y[alpha, beta] = X
    return Y


def _unconfuse(Y: np.ndarray, k: np.ndarray) -> np.ndarray:
    H, W, _ = Y.shape
    alpha, beta = _perm(H, W, k)
    return Y[alpha, beta]


def _diffuse(Y: np.ndarray, ks_round: list[np.ndarray], bnd, seed_from: np.ndarray | None = None) -> np.ndarray:
    """Eq. 3 per subframe as an XOR scan of d = b xor (y + b), the first byte
    also XORed with s_d = the last byte of subframe (i + 1) mod n of
    ``seed_from`` (the confused frame Y unless a mutation says otherwise)."""
    n = len(bnd) - 1
    y = Y.ravel()
    src = y if seed_from is None else seed_from.ravel()
    out = np.empty_like(y)
    for i in range(n):
        b = ks_round[i]
        d = b ^ ((y[bnd[i]:bnd[i + 1]].astype(np.uint16) + b) & 255).astype(np.uint8)
        d[0] ^= src[bnd[(i + 1) % n + 1] - 1]
        out[bnd[i]:bnd[i + 1]] = np.bitwise_xor.accumulate(d)
    return out.reshape(Y.shape)


def _undiffuse(Xc: np.ndarray, ks_round: list[np.ndarray], bnd) -> np.ndarray:
    """Eq. 4: y_q = (b xor c_q xor c_{q-1}) - b inside each subframe, then the
    first bytes with the seed recovered from the next subframe's last byte."""
    n = len(bnd) - 1
    c = Xc.ravel()
    y = np.empty_like(c)
    for i in range(n):
        b = ks_round[i]
        seg = c[bnd[i]:bnd[i + 1]]
        y[bnd[i] + 1:bnd[i + 1]] = ((b[1:] ^ seg[1:] ^ seg[:-1]).astype(np.int16) - b[1:]) & 255
    for i in range(n):
        b0 = int(ks_round[i][0])
        s = int(y[bnd[(i + 1) % n + 1] - 1])
        y[bnd[i]] = ((b0 ^ int(c[bnd[i]]) ^ s) - b0) & 255
    return y.reshape(Xc.shape)


def _compose_encrypt(X, sc_list, streams, H, W, C, n, r, orc, mutation=None):
    """Alg. 1 / Alg. 2 for consecutive frames X[f]: frame f uses s_c = sc_list[f]
    and bytes [f r S_i, (f + 1) r S_i) of subframe i's stream, round j the
    slice [j S_i, (j + 1) S_i) of those; each round confusion then diffusion."""
    bnd = _bounds(H, W, C, n)
    S = [bnd[i + 1] - bnd[i] for i in range(n)]
    out = []
    for f in range(X.shape[0]):
        sc = sc_list[f + 1] if mutation == "next_sc" else sc_list[f]
        k = _ktable(H, sc, orc)
        Z = X[f].copy()
        for j in range(r):
            jj = r - 1 - j if mutation == "reverse_rounds" else j
            if mutation == "per_frame_cut":  # the frame's bytes cut subframe-major instead of per subframe
                flat = np.concatenate([streams[i][f * r * S[i]:(f + 1) * r * S[i]] for i in range(n)])
                off = sum(S)
                ks_round = [flat[jj * off + bnd[i]: jj * off + bnd[i + 1]] for i in range(n)]
            else:
                ks_round = [streams[i][(f * r + jj) * S[i]:(f * r + jj + 1) * S[i]] for i in range(n)]
            if mutation == "diffuse_first":
                Z = _confuse(_diffuse(Z, ks_round, bnd), k)
            else:
                Y = _confuse(Z, k)
                if mutation == "seed_after_diffusion":
                    Z = _diffuse(Y, ks_round, bnd, seed_from=_diffuse(Y, ks_round, bnd))
                else:
                    Z = _diffuse(Y, ks_round, bnd)
        out.append(Z)
    return np.stack(out)


def _compose_decrypt(Zc, sc_list, streams, H, W, C, n, r, orc):
    bnd = _bounds(H, W, C, n)
    S = [bnd[i + 1] - bnd[i] for i in range(n)]
    out = []
    for f in range(Zc.shape[0]):
        k = _ktable(H, sc_list[f], orc)
        Z = Zc[f].copy()
        for j in range(r - 1, -1, -1):
            ks_round = [streams[i][(f * r + j) * S[i]:(f * r + j + 1) * S[i]] for i in range(n)]
            Z = _unconfuse(_undiffuse(Z, ks_round, bnd), k)
        out.append(Z)
    return np.stack(out)


# --------------------------------------------------------------- exact integer case

def _exact_setup(orc, H, W, C, n, r, F, seed):
    """A PLCM context whose PRBG_m and every PRBG_a^i run at p = 1/4 from
    dyadic starting values, and the exact streams and s_c of its frames."""
    rng = np.random.default_rng(seed)
    Xm = [int(rng.integers(1 << 40, 1 << 52)) | 1 for _ in range(2)]
    main = _exact_pair_stream(Xm[0], Xm[1], 6 * (4 * n + F + 1))
    groups = _groups(main)
    sc_list = [1 + groups[4 * n + f] % 65536 for f in range(F + 1)]
    enc = orc.OracleCipher(orc.PLCM, [Xm[0] / 2 ** 52, 0.25, Xm[1] / 2 ** 52, 0.25], H, W, C, n, r)
    dec = orc.OracleCipher(orc.PLCM, [Xm[0] / 2 ** 52, 0.25, Xm[1] / 2 ** 52, 0.25], H, W, C, n, r)
    # the key schedule's closed form (Alg. 1): P_m from groups 4i .. 4i + 3
    for i in range(n):
        prm = enc.sub_params(i)
        assert prm[0] == _unit(groups[4 * i]) and prm[1] == 0.05 + 0.4 * _unit(groups[4 * i + 1])
        assert prm[2] == _unit(groups[4 * i + 2]) and prm[3] == 0.05 + 0.4 * _unit(groups[4 * i + 3])
    bnd = _bounds(H, W, C, n)
    streams = []
    for i in range(n):
        X1, X2 = (int(rng.integers(1 << 44, 1 << 52)) | 1 for _ in range(2))
        for c in (enc, dec):
            c.set_sub_params(i, [X1 / 2 ** 52, 0.25, X2 / 2 ** 52, 0.25])
        streams.append(_exact_pair_stream(X1, X2, F * r * (bnd[i + 1] - bnd[i])))
    return enc, dec, sc_list, streams


@pytest.mark.parametrize("H,W,C,n,r", [(4, 5, 3, 5, 5), (4, 5, 3, 5, 2), (5, 5, 3, 7, 5), (6, 7, 1, 3, 1),
                                       (3, 4, 4, 3, 5), (5, 6, 3, 1, 5)])
def test_frame_loop_exact_integer_orbits(orc, H, W, C, n, r):
    """Every keystream byte, every s_c and so every ciphertext byte of 4 frames
    follows from exact integer orbits (p = 1/4, dyadic x0): the oracle's
    encrypt and decrypt equal the composition byte for byte.  (At p = 1/4 an
    orbit loses two low bits per step, so the later groups of PRBG_m give
    s_c = 1; with n = 1 the frames' s_c come from early, full groups.)"""
    F = 4
    enc, dec, sc_list, streams = _exact_setup(orc, H, W, C, n, r, F, seed=H * 100 + n * 10 + r)
    assert any(s[:r * 12].any() for s in streams)  # the orbits are still alive in the first frames
    X = synth.uniform_frames(F, H, W, C, seed=7 + n)
    exp = _compose_encrypt(X, sc_list, streams, H, W, C, n, r, orc)
    got = enc.encrypt(X)
    assert np.array_equal(got, exp)
    # decryption of arbitrary bytes (not only of this ciphertext) follows Eq. 4 / Eq. 2
    Z = synth.uniform_frames(F, H, W, C, seed=9 + n)
    assert np.array_equal(dec.decrypt(Z), _compose_decrypt(Z, sc_list, streams, H, W, C, n, r, orc))


# --------------------------------------------------------------- general keys, pinned parts

_PAIR = {0: 0, 1: 1, 2: 3}  # map kind -> PRBG kind of its subframe pairs
_MAIN = {0: 0, 1: 2, 2: 3}  # map kind -> PRBG kind of PRBG_m


def _schedule_from_stream(orc, kind, key, n, F):
    """Alg. 1 from PRBG_m's own byte stream (the pinned PRBG): the subframe
    parameters and the s_c of frames 0 .. F."""
    per = 6 if kind == 1 else 4
    mkey = list(key) if kind != 1 else [key[0], key[2], key[1]]  # (x0, mu, y0) -> state (x, y, mu)
    groups = _groups(np.frombuffer(orc.prbg_bytes(_MAIN[kind], mkey, 6 * (per * n + F + 1)), dtype=np.uint8))
    params = []
    for i in range(n):
        u = [_unit(U) for U in groups[per * i: per * (i + 1)]]
        if kind == 0:
            params.append([u[0], 0.05 + 0.4 * u[1], u[2], 0.05 + 0.4 * u[3]])
        elif kind == 2:
            params.append([u[0], 3.9 + 0.1 * u[1], u[2], 3.9 + 0.1 * u[3]])
        else:
            params.append([u[0], u[1], 0.44 + 0.49 * u[2], u[3], u[4], 0.44 + 0.49 * u[5]])
    sc_list = [1 + groups[per * n + f] % 65536 for f in range(F + 1)]
    return params, sc_list


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("H,W,C,n,r", [(16, 20, 3, 7, 5), (9, 11, 3, 5, 2), (12, 12, 1, 9, 1), (7, 13, 4, 3, 5)])
def test_frame_loop_from_pinned_parts(orc, kind, H, W, C, n, r):
    """The same composition for every map with general keys: PRBG_m's stream
    gives P_m and s_c, each subframe's stream is the pinned PRBG from those
    parameters, and 4 consecutive frames equal the oracle's encrypt and
    decrypt byte for byte."""
    F = 4
    key = synth.key_for_seed(kind, 500 + n)
    params, sc_list = _schedule_from_stream(orc, kind, key, n, F)
    bnd = _bounds(H, W, C, n)
    streams = [np.frombuffer(orc.prbg_bytes(_PAIR[kind], params[i], F * r * (bnd[i + 1] - bnd[i])), dtype=np.uint8)
               for i in range(n)]
    enc = orc.OracleCipher(kind, key, H, W, C, n, r)
    X = synth.smooth_clip(F, H, W, C, seed=3) if C == 3 else synth.uniform_frames(F, H, W, C, seed=3)
    assert np.array_equal(enc.encrypt(X), _compose_encrypt(X, sc_list, streams, H, W, C, n, r, orc))
    dec = orc.OracleCipher(kind, key, H, W, C, n, r)
    Z = synth.uniform_frames(F, H, W, C, seed=4)
    assert np.array_equal(dec.decrypt(Z), _compose_decrypt(Z, sc_list, streams, H, W, C, n, r, orc))


@pytest.mark.parametrize("mutation", ["reverse_rounds", "per_frame_cut", "diffuse_first", "next_sc",
                                      "seed_after_diffusion"])
def test_composition_slips_change_the_ciphertext(orc, mutation):
    """Each plausible slip in the frame loop gives different bytes, so the two
    tests above would fail on it: round slices taken in reverse or cut from
    the frame's bytes subframe-major, diffusion before confusion, the next
    frame's s_c, the diffusion seed read after diffusion."""
    H, W, C, n, r, F = 9, 11, 3, 5, 3, 2
    key = synth.key_for_seed(0, 505)
    params, sc_list = _schedule_from_stream(orc, 0, key, n, F)
    bnd = _bounds(H, W, C, n)
    streams = [np.frombuffer(orc.prbg_bytes(0, params[i], F * r * (bnd[i + 1] - bnd[i])), dtype=np.uint8)
               for i in range(n)]
    X = synth.uniform_frames(F, H, W, C, seed=5)
    ref = orc.OracleCipher(0, key, H, W, C, n, r).encrypt(X)
    assert np.array_equal(ref, _compose_encrypt(X, sc_list, streams, H, W, C, n, r, orc))
    bad = _compose_encrypt(X, sc_list, streams, H, W, C, n, r, orc, mutation=mutation)
    assert not np.array_equal(bad, ref)
