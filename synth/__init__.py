"""Seeded synthetic inputs and workload shapes shared by the oracle tests, the CUDA tests
and the benchmark.  Holds no arithmetic of the method: only random draws (numpy
PCG64 generators seeded per use), bit packing of spin configurations, and the
workload definitions (lattice sizes, rates, sample counts) as plain data.
"""
from dataclasses import dataclass, field, asdict
import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    extent: tuple            # lattice extent: (N,) chain or (Lx, Ly) square, open boundaries
    J: float
    alpha: float
    h: float
    kappa: float             # decay rate of every site
    gamma: float             # dephasing rate of every site
    ansatz: str              # "jastrow" or "rbm"
    n_hidden: int
    ns: int                  # samples (= Markov chains) per trajectory
    ntraj: int
    dt: float
    n_steps: int
    scheme: str              # "heun" or "midpoint"
    eps: float = 1e-4        # diagonal shift of the regularised solve
    n_sweep: int = 2         # Metropolis sweeps (N proposals each) per evaluation
    pbc: bool = False
    kac: bool = False
    lj_d: int = 0            # tie distance of the "lj" ansatz (LJPHd; 0 = LJH)

    @property
    def n(self):
        return int(np.prod(self.extent))

    def to_dict(self):
        return asdict(self)


# The five benchmark workloads: long-range transverse-field Ising quenches from the
# coherent state along +x with local decay (and dephasing), shaped like the paper's.
WORKLOADS = {
    "chain8_jastrow": Workload("chain8_jastrow", (8,), 1.0, 1.5, 1.0, 0.1, 0.0, "jastrow", 0,
                               1024, 16, 0.01, 100, "heun"),
    "chain64_jastrow": Workload("chain64_jastrow", (64,), 1.0, 1.5, 1.0, 0.1, 0.05, "jastrow", 0,
                                4096, 256, 0.005, 400, "midpoint"),
    "square10_jastrow": Workload("square10_jastrow", (10, 10), 1.0, 3.0, 0.5, 0.05, 0.0, "jastrow", 0,
                                 8192, 512, 0.005, 200, "midpoint"),
    "chain64_rbm": Workload("chain64_rbm", (64,), 1.0, 1.5, 1.0, 0.1, 0.0, "rbm", 128,
                            8192, 128, 0.005, 200, "midpoint"),
    "square16_rbm": Workload("square16_rbm", (16, 16), 1.0, 1.5, 1.0, 0.1, 0.0, "rbm", 256,
                             4096, 64, 0.005, 200, "midpoint"),
}

# The paper's large-N setups with the tied ansatz LJPH1 (periodic ring, alpha = 1 with the Kac
# factor, the LITF sign: couplings -J/(K r), field -h), 400 trajectories to t = 0.8.
PAPER_WORKLOADS = {
    "ring100_ljph1": Workload("ring100_ljph1", (100,), -1.0, 1.0, -1.07, 0.27, 0.0, "lj", 0,
                              4096, 400, 0.005, 160, "midpoint", pbc=True, kac=True, lj_d=1),
    "ring160_ljph1": Workload("ring160_ljph1", (160,), -1.0, 1.0, 0.0, 0.1, 0.0, "lj", 0,
                              4096, 400, 0.005, 160, "midpoint", pbc=True, kac=True, lj_d=1),
}


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def random_theta(seed, ntraj, P, scale=0.05):
    """Complex parameters with independent N(0, scale^2) real and imaginary parts."""
    g = rng(seed)
    return (g.normal(0, scale, (ntraj, P)) + 1j * g.normal(0, scale, (ntraj, P)))


def random_spins(seed, ntraj, ns, n):
    """Uniform i.i.d. sigma in {-1, +1}, shape (ntraj, ns, n), int8."""
    g = rng(seed)
    return np.where(g.integers(0, 2, (ntraj, ns, n)) == 1, 1, -1).astype(np.int8)


def random_normals(seed, shape, scale=1.0):
    return rng(seed).normal(0, scale, shape)


def pack_spins(sig):
    """(..., n) sigma in {-1,+1} -> (..., ceil(n/64)) uint64; bit j of word j//64 set <=> +1."""
    sig = np.asarray(sig)
    n = sig.shape[-1]
    nw = (n + 63) // 64
    out = np.zeros(sig.shape[:-1] + (nw,), dtype=np.uint64)
    for j in range(n):
        out[..., j // 64] |= (sig[..., j] > 0).astype(np.uint64) << np.uint64(j % 64)
    return out


def unpack_spins(words, n):
    words = np.asarray(words, dtype=np.uint64)
    j = np.arange(n)
    bits = (words[..., j // 64] >> (j % 64).astype(np.uint64)) & np.uint64(1)
    return np.where(bits == 1, 1, -1).astype(np.int8)
