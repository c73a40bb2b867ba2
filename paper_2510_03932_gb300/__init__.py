"""GB300-native evaluator for trapezoidal direct transcriptions of optimal control problems.

Importing the package is cheap; the CUDA library is loaded on first use by `ocp`.
"""
