"""GB300-native CKKS homomorphic linear transformation (TH-BSGS and baselines).

The compute path is the C-ABI library built from csrc/ (hand-written CUDA for
sm_103a); `binding` marshals arguments to it.  `synth` holds the seeded input
generators.  Importing the package does not load the CUDA library.
"""
__all__ = ["synth", "binding"]
