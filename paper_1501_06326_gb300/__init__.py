"""GB300-native Aggregate Risk Analysis (ARA) with secondary uncertainty.

The package is deliberately light at import time: ``synth`` (seeded input
generators) imports only numpy, and the CUDA binding lives in ``ara`` and is
loaded on first use, so that importing the generators never loads the CUDA
library.
"""

__all__ = ["synth", "ara"]
