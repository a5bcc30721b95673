"""B300-native event-based Monte Carlo transport and macroscopic cross-section
lookup (the computation autotuned in arXiv 2402.09222, Sec. 5.1).

    from paper_2402_09222_b300 import mcx, synth
    prob = synth.config3_problem(n_histories=100_000)
    p = mcx.make_problem(prob, precision=mcx.FP32, hash_bins=4000)
    p.set_tuning(mode=mcx.QUEUED, sort_period=4).run(particles_in_flight=1_000_000, seed=7)
    tallies = p.tallies()

`mcx` is the binding of the CUDA library (imported on demand: it raises if
libmcx.so is missing); `synth` generates the seeded synthetic inputs.
"""
import importlib

__all__ = ["mcx", "synth", "tuner"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
