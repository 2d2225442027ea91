"""Seeded synthetic inputs for the CHESSFAD hot path.

This module is the one piece shared by the CUDA path's callers and the oracle:
it draws inputs and nothing else -- none of the chunked-hDual arithmetic lives
here.  The only arithmetic is the definition of a Fletcher-Powell instance,
E_m = sum_j (A_mj sin alpha_j + B_mj cos alpha_j), which makes alpha a zero of
the residuals.

Every draw uses ``numpy.random.Generator(PCG64(seed))`` in a fixed order.
The paper measures on "1K points CPU / 0.5M points GPU" of the same three
functions (Sec. VII) and names no dataset; these seeded draws stand in for it.

Named workloads (function, n, batch, seed):

* ``rosenbrock_n16``  Rosenbrock, n=16, 4096 points, x~U[-2,2], v~U[-1,1], seed 0
* ``ackley_n64``      Ackley, n=64, 65536 points, x~U[-5,5], v~U[-1,1], seed 1
* ``fletcher_powell_n32``  Fletcher-Powell, n=32, 16384 points: alpha~U[-pi,pi]^32,
  A, B ~ U[-100,100]^{32x32}, x~U[-pi,pi], v~U[-1,1], seed 2
* ``rosenbrock_n256`` Rosenbrock, n=256, 1024 points, seed 3
* ``ragged_100k``     100000 requests, function uniform over the three,
  n = round(exp(U[ln 2, ln 512])), x by the function's range, v~U[-1,1];
  one alpha (512), A, B (512x512) whose leading n x n block serves size n,
  and E^(n) per distinct n; seed 4
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ROSENBROCK, ACKLEY, FLETCHER_POWELL = 0, 1, 2
# A test function of the extended operator set (division, abs, log, tanh,
# tan, pow and a comparison), evaluated through the user-function interface;
# the library has no built-in id for it.
MIX = 3
FN_NAMES = {ROSENBROCK: "rosenbrock", ACKLEY: "ackley", FLETCHER_POWELL: "fletcher_powell", MIX: "mix"}
X_RANGE = {ROSENBROCK: (-2.0, 2.0), ACKLEY: (-5.0, 5.0), FLETCHER_POWELL: (-math.pi, math.pi), MIX: (-2.0, 2.0)}


@dataclass
class FPInstance:
    """Fletcher-Powell parameters shared by a whole batch (FP64)."""
    alpha: np.ndarray
    A: np.ndarray
    B: np.ndarray
    E: np.ndarray

    def leading(self, n: int) -> "FPInstance":
        """The size-n instance that uses the leading n x n block of A, B."""
        A = np.ascontiguousarray(self.A[:n, :n])
        B = np.ascontiguousarray(self.B[:n, :n])
        return FPInstance(self.alpha[:n].copy(), A, B, fp_rhs(A, B, self.alpha[:n]))


def fp_rhs(A: np.ndarray, B: np.ndarray, alpha: np.ndarray) -> np.ndarray:
    """E_m = sum_j A_mj sin(alpha_j) + B_mj cos(alpha_j): the instance's
    right-hand side, chosen so that x = alpha zeroes every residual."""
    return A @ np.sin(alpha) + B @ np.cos(alpha)


def draw_fp_instance(rng: np.random.Generator, n: int) -> FPInstance:
    alpha = rng.uniform(-math.pi, math.pi, n)
    A = rng.uniform(-100.0, 100.0, (n, n))
    B = rng.uniform(-100.0, 100.0, (n, n))
    return FPInstance(alpha, A, B, fp_rhs(A, B, alpha))


@dataclass
class Batch:
    """A dense batch: x, v are [batch, n] FP64; fp holds Fletcher-Powell data."""
    name: str
    fn: int
    n: int
    x: np.ndarray
    v: np.ndarray
    fp: FPInstance | None = None
    seed: int = 0

    @property
    def batch(self) -> int:
        return self.x.shape[0]


def make_batch(fn: int, n: int, batch: int, seed: int, name: str | None = None) -> Batch:
    """Draw a batch in the fixed order: [alpha, A, B for Fletcher-Powell], x, v."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fp = draw_fp_instance(rng, n) if fn == FLETCHER_POWELL else None
    lo, hi = X_RANGE[fn]
    x = rng.uniform(lo, hi, (batch, n))
    v = rng.uniform(-1.0, 1.0, (batch, n))
    return Batch(name or f"{FN_NAMES[fn]}_n{n}_b{batch}_s{seed}", fn, n, x, v, fp, seed)


WORKLOADS = {
    "rosenbrock_n16": (ROSENBROCK, 16, 4096, 0),
    "ackley_n64": (ACKLEY, 64, 65536, 1),
    "fletcher_powell_n32": (FLETCHER_POWELL, 32, 16384, 2),
    "rosenbrock_n256": (ROSENBROCK, 256, 1024, 3),
}


def workload(name: str, batch: int | None = None) -> Batch:
    """A named workload; ``batch`` keeps only the first rows of the full draw
    (same values as the full-size workload, so samples stay comparable)."""
    fn, n, full, seed = WORKLOADS[name]
    b = make_batch(fn, n, full, seed, name)
    if batch is not None and batch < full:
        b = Batch(name, fn, n, b.x[:batch].copy(), b.v[:batch].copy(), b.fp, seed)
    return b


@dataclass
class Ragged:
    """Packed uneven batch: request q has function fns[q] and size ns[q]; its
    x, v, out occupy [offs[q], offs[q] + ns[q]) of the packed arrays.  A
    Fletcher-Powell request of size n uses the leading n x n block of the
    shared A, B (leading dimension ``ld``) and E at Epack[eoffs[q]:][:n]."""
    fns: np.ndarray
    ns: np.ndarray
    offs: np.ndarray
    xpack: np.ndarray
    vpack: np.ndarray
    fp: FPInstance
    Epack: np.ndarray
    eoffs: np.ndarray
    e_of_n: dict = field(default_factory=dict)

    @property
    def nreq(self) -> int:
        return len(self.fns)

    @property
    def ld(self) -> int:
        return self.fp.A.shape[1]

    def subset(self, idx) -> "Ragged":
        """Requests idx (in that order), repacked; FP data shared."""
        idx = np.asarray(idx)
        fns = self.fns[idx]
        ns = self.ns[idx]
        offs = np.zeros(len(idx), dtype=np.int64)
        if len(idx):
            offs[1:] = np.cumsum(ns[:-1])
        total = int(ns.sum())
        xp = np.empty(total)
        vp = np.empty(total)
        for q, src in enumerate(idx):
            o, n = self.offs[src], self.ns[src]
            xp[offs[q]:offs[q] + n] = self.xpack[o:o + n]
            vp[offs[q]:offs[q] + n] = self.vpack[o:o + n]
        return Ragged(fns, ns, offs, xp, vp, self.fp, self.Epack, self.eoffs[idx].copy(), self.e_of_n)


def make_ragged(nreq: int = 100000, seed: int = 4, nmax: int = 512) -> Ragged:
    """Draw order: fns, ns, alpha (nmax), A, B (nmax x nmax), x uniforms, v."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fns = rng.integers(0, 3, size=nreq).astype(np.int32)
    ns = np.rint(np.exp(rng.uniform(math.log(2.0), math.log(nmax), size=nreq))).astype(np.int32)
    ns = np.clip(ns, 2, nmax).astype(np.int32)
    fp = draw_fp_instance(rng, nmax)
    offs = np.zeros(nreq, dtype=np.int64)
    if nreq:
        offs[1:] = np.cumsum(ns[:-1].astype(np.int64))
    total = int(ns.astype(np.int64).sum())
    u = rng.uniform(0.0, 1.0, total)
    vpack = rng.uniform(-1.0, 1.0, total)
    lo = np.empty(total)
    hi = np.empty(total)
    req_of = np.repeat(np.arange(nreq), ns)
    for f, (a, b) in X_RANGE.items():
        sel = fns[req_of] == f
        lo[sel], hi[sel] = a, b
    xpack = lo + (hi - lo) * u
    # E^(n) for every distinct n used by a Fletcher-Powell request.
    e_of_n: dict[int, int] = {}
    chunks = []
    pos = 0
    for n in sorted(set(int(k) for k in ns[fns == FLETCHER_POWELL])):
        e = fp_rhs(fp.A[:n, :n], fp.B[:n, :n], fp.alpha[:n])
        e_of_n[n] = pos
        chunks.append(e)
        pos += n
    Epack = np.concatenate(chunks) if chunks else np.zeros(1)
    eoffs = np.array([e_of_n.get(int(n), 0) if f == FLETCHER_POWELL else 0 for f, n in zip(fns, ns)],
                     dtype=np.int64)
    return Ragged(fns, ns, offs, xpack, vpack, fp, Epack, eoffs, e_of_n)


def round_to_f32(a: np.ndarray) -> np.ndarray:
    """Inputs of the compensated-FP32 path are float; the oracle receives the
    same rounded values (so input rounding is not charged to the method)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)
