"""CPU FP64 oracle for random-circuit amplitudes.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of ``bench.py``
may import this package.  The CUDA path in ``paper_1905_00444_gb300`` never imports
it, and it never imports the CUDA path: the two share no code.  The only common
module is ``rqc_inputs`` (seeded circuit and bitstring generators, no method
arithmetic).

What it computes is the plain definition of the quantity the method reaches
exactly: the amplitude <x| C |0^n> of a circuit C (the paper's RCS problem
statement, Fig. 1 "Probability(circuit, s)", and its tensor-network form, Sec. II).
Independent routes, each pinned by ``tests/test_oracle_*.py``:

* ``dense``        -- full 2^n x 2^n unitary from Kronecker products (n <= 10);
* ``statevector``  -- gate-by-gate state vector, complex128 (n <= ~24);
* ``network``      -- time-first folding of each grid site into one tensor (Sec. III,
                      Fig. 3) with each diagonal two-qubit gate as a dimension-2 bond,
                      then a row-major sweep of labelled ``np.tensordot`` calls; also
                      cuts (Sec. III.A) by fixing bond values;
* ``stabilizer``   -- Aaronson-Gottesman tableau, exact |amp|^2 of Clifford circuits at
                      any grid size (pins full-size runs by a property);
* ``gradient``     -- gate gradients by linearity of the amplitude in each gate;
* ``primitives``   -- the single contraction step (TTGT, Sec. III.E), permutation and
                      the flop count of Eq. 1, written as their definitions;
* ``sampling``     -- frugal rejection sampling over fast-sampling batches (Sec. III.B),
                      the bitstring assembly x1 u x2 and the linear cross-entropy
                      fidelity used to check noisy (path-fraction) sampling (Sec. III.C).

Parity status: every function above is pinned by closed forms, brute force or an
independent route; none is "parity unpinned".
"""
from . import dense, statevector, network, stabilizer, gradient, primitives, sampling  # noqa: F401
