"""CPU FP64 oracle for the tensor-network amplitude path.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check of the package entry
module and the CPU-baseline leg of the benchmark may import anything here; the
product path never calls it and shares no code with it (the CUDA path has its
own network builder, path finder, kernels and sampler).  Inputs come from the
seeded generators in ``workloads``.

Modules:
  statevector  -- O1: brute-force statevector / density-matrix simulation
                  (the plain definition <x| U |0...0> of Eq. ampl_calc and
                  rho -> sum_k A_k rho A_k^dagger of Eq. kraus_sum).
  tn           -- O2: a plain pairwise tensor-network contractor with its own
                  builder (Sec. 3.1), projection (Sec. 3.1.1), greedy order and
                  index slicing (Sec. 3.1), usable beyond statevector sizes.
  noise        -- the stochastic Kraus-trajectory estimator and its
                  counter-based SplitMix64 draws.
  contraction  -- the pairwise complex contraction of two all-dimension-2
                  tensors over their shared labels (one step of Sec. 3.1).
  mlp          -- FP64 reference of the path cost model's MLP (forward,
                  backward, Adam).
  golden       -- readers of the stored contraction trees and expected
                  values (tests/golden).

O2 also evaluates marginal wave-function slices (Sec. 4.4: qubits left open),
the doubled density-matrix network of Sec. 3.3 (exact noisy probabilities),
and follows a contraction tree given over groups of circuit tensors, with its
own slicing, so that it can contract the 36-qubit benchmark circuit.
"""
