"""FP64 CPU oracle for joint-cut HSF simulation (test infrastructure only).

Importable by the tests, the smoke check and the benchmark's CPU-baseline leg only;
the product library never imports it."""
from .hsf_oracle import *  # noqa: F401,F403
from .hsf_oracle import (apply_gate, block_qubits, block_unitary, circuit_unitary_bruteforce,
                         classify, decompose_blocks, embed_bruteforce, execution_order,
                         fd_gradient, gate_derivative, gate_matrix, hsf_amplitudes,
                         loss_from_amplitudes, schmidt_decompose, schmidt_reconstruct,
                         schrodinger)
