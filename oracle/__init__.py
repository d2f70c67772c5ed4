"""CPU oracle of the driving-simulator step (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
package.  It is independent of the CUDA library: its arithmetic is in
``oracle.cpp`` (brute force, templated on float/double) and in
``gradient.py`` (the gradient of the rollout loss by PyTorch autograd in
float64).  See ``oracle.cpp`` for the paper passages each part follows.
"""
from .oracle import Oracle, OracleConfig, build_oracle, load_oracle  # noqa: F401
