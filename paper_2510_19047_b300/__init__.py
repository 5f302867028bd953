"""B300-native time-frequency semi-coherent statistic (arXiv:2510.19047).

``binding.TFS`` is the entry point: a context on one GPU with ``load_tf_data``,
``set_noise_weights``, ``eval_statistic``, ``grad_statistic`` (the C ABI of
``include/tfs.h``). ``synth`` makes seeded synthetic workloads.
"""
__all__ = ["binding", "synth", "build"]
