"""Philox4x32-10 counter-based generator and the draws the otVMC method makes.

Test infrastructure (oracle side).  This module is an independent restatement of the
Philox4x32 generator from its published definition (Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11, section 5): ten rounds, each
multiplying two of the four 32-bit counter words by fixed odd constants, XOR-ing the
high halves of the products with the other two words and the key, and bumping the key
by two Weyl constants between rounds.  The CUDA library has its own implementation;
the two share no code.

Draws of the method (conventions shared with the CUDA library as an interface, not as
code; the paper only says the increments are Wiener increments of variance dt and that
sampling is by Metropolis, Eq. 2 and the otVMC procedure):

* key = (seed mod 2^32, seed >> 32)
* Wiener increments (Eq. 2, Delta W_n ~ N(0, dt)):
    counter = (n // 4, step, trajectory, TAG_NOISE << 28); the four 32-bit words give
    two Box-Muller pairs: n % 4 in {0, 1} from words (0, 1), {2, 3} from words (2, 3).
* Metropolis proposals (two per counter):
    counter = (p // 2, chain, trajectory, (TAG_SAMPLE << 28) | (eval_index mod 2^28));
    proposal p uses words (2*(p%2), 2*(p%2)+1): site = (w0 * N) >> 32, u = (w1 + 0.5) 2^-32.
* Initial configurations (two 64-bit words per counter):
    counter = (q, chain, trajectory, TAG_INIT << 28); spin word 2q = w0 | w1 << 32,
    word 2q+1 = w2 | w3 << 32; bit j of word j // 64 set <=> sigma_j = +1.
"""
import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)

TAG_SAMPLE = 1
TAG_NOISE = 2
TAG_INIT = 3


def philox4x32_10(counter, key):
    """Philox4x32 with 10 rounds.

    counter: integer array (..., 4) of 32-bit words; key: integer array (..., 2).
    Returns uint32 array (..., 4).  Broadcasting over the leading axes.
    """
    ctr = np.asarray(counter, dtype=np.uint64) & MASK32
    k = np.asarray(key, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = ctr[..., 0], ctr[..., 1], ctr[..., 2], ctr[..., 3]
    k0, k1 = k[..., 0], k[..., 1]
    for r in range(10):
        if r > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0          # < 2^64: exact in uint64
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def seed_key(seed):
    seed = int(seed)
    return np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)


def uniform_open(w):
    """32-bit word -> uniform double in (0, 1): (w + 1/2) 2^-32 (exact in FP64)."""
    return (np.asarray(w, dtype=np.float64) + 0.5) * (2.0 ** -32)


def box_muller(u0, u1):
    """Two independent standard normals from two uniforms in (0, 1)."""
    rad = np.sqrt(-2.0 * np.log(u0))
    ang = 2.0 * np.pi * u1
    return rad * np.cos(ang), rad * np.sin(ang)


def wiener_increments(seed, traj_ids, step, n_ops, dt):
    """Delta W[t, n] ~ N(0, dt), i.i.d. over trajectories and jump operators (Eq. 2).

    One draw per trajectory and step, shared by the predictor and corrector stages
    (App. C applies both stages with the same Delta W_i).
    """
    traj_ids = np.asarray(traj_ids, dtype=np.uint64)
    nq = (n_ops + 3) // 4
    q = np.arange(nq, dtype=np.uint64)
    ctr = np.zeros((len(traj_ids), nq, 4), dtype=np.uint64)
    ctr[..., 0] = q[None, :]
    ctr[..., 1] = np.uint64(step)
    ctr[..., 2] = traj_ids[:, None]
    ctr[..., 3] = np.uint64(TAG_NOISE << 28)
    w = philox4x32_10(ctr, seed_key(seed))
    u = uniform_open(w)
    z0, z1 = box_muller(u[..., 0], u[..., 1])
    z2, z3 = box_muller(u[..., 2], u[..., 3])
    z = np.stack([z0, z1, z2, z3], axis=-1).reshape(len(traj_ids), 4 * nq)
    return np.sqrt(dt) * z[:, :n_ops]


def proposal_draws(seed, traj_id, n_chains, eval_index, p, n_sites, chain_ids=None):
    """Site index and acceptance uniform of proposal p for every chain of one trajectory
    (chains 0..n_chains-1, or the given chain ids)."""
    ids = np.arange(n_chains, dtype=np.uint64) if chain_ids is None else np.asarray(chain_ids, dtype=np.uint64)
    ctr = np.zeros((len(ids), 4), dtype=np.uint64)
    ctr[:, 0] = np.uint64(p // 2)
    ctr[:, 1] = ids
    ctr[:, 2] = np.uint64(traj_id)
    ctr[:, 3] = np.uint64((TAG_SAMPLE << 28) | (int(eval_index) & 0x0FFFFFFF))
    w = philox4x32_10(ctr, seed_key(seed)).astype(np.uint64)
    h = 2 * (p % 2)
    site = ((w[:, h] * np.uint64(n_sites)) >> np.uint64(32)).astype(np.int64)
    u = uniform_open(w[:, h + 1])
    return site, u


def initial_spins(seed, traj_id, n_chains, n_sites):
    """I.i.d. uniform configurations, sigma in {-1, +1}, shape (n_chains, n_sites).

    At theta = 0 both ansaetze describe the coherent state along +x, whose |psi|^2 is
    uniform over the sigma^z basis, so these are exact samples with no burn-in.
    """
    n_words = (n_sites + 63) // 64
    nq = (n_words + 1) // 2
    ctr = np.zeros((n_chains, nq, 4), dtype=np.uint64)
    ctr[..., 0] = np.arange(nq, dtype=np.uint64)[None, :]
    ctr[..., 1] = np.arange(n_chains, dtype=np.uint64)[:, None]
    ctr[..., 2] = np.uint64(traj_id)
    ctr[..., 3] = np.uint64(TAG_INIT << 28)
    w = philox4x32_10(ctr, seed_key(seed)).astype(np.uint64)
    words = np.empty((n_chains, 2 * nq), dtype=np.uint64)
    words[:, 0::2] = w[..., 0] | (w[..., 1] << np.uint64(32))
    words[:, 1::2] = w[..., 2] | (w[..., 3] << np.uint64(32))
    j = np.arange(n_sites)
    bits = (words[:, j // 64] >> (j % 64).astype(np.uint64)) & np.uint64(1)
    return np.where(bits == 1, 1, -1).astype(np.int8)
