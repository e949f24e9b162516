"""B300-native (sm_103a) vectorised training of many per-object MLP neural
fields, after vMAP (Kong et al., CVPR 2023, section 3.2 "Vectorised Training").

    from paper_2302_01838_b300.api import VMap      # C-ABI wrapper (needs the built .so)
    from paper_2302_01838_b300 import scenes        # seeded synthetic inputs
"""
