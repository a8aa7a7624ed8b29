"""The seeded tomography inputs: shapes, ranges and determinism (Sec. 4.1
stand-ins)."""
import numpy as np

import synth.tomo as st


def test_stations_are_distinct_interior_nodes_and_seeded():
    cfg = st.tomo_config("tomo_uk")
    sta = st.stations(cfg)
    assert sta.shape == (61,) and len(set(sta.tolist())) == 61
    i, j = np.divmod(sta, cfg.nx)
    assert i.min() >= 1 and i.max() <= cfg.ny - 2 and j.min() >= 1 and j.max() <= cfg.nx - 2
    assert np.array_equal(sta, st.stations(cfg))
    assert not np.array_equal(sta, st.stations(cfg, seed=4))


def test_maps_lie_inside_the_prior_and_data_shapes_agree():
    cfg = st.tomo_config("tomo_uk")
    v = st.true_group_velocity(cfg)
    assert v.shape == (40, 37) and v.min() >= 1.8 and v.max() <= 4.5
    X = st.particles_from_prior(cfg, 7)
    assert X.shape == (7, cfg.d) and X.min() >= cfg.vmin and X.max() <= cfg.vmax
    S = st.smooth_particles(cfg, 3)
    assert S.min() >= 1.7 and S.max() <= 4.6
    sig = st.pair_sigma(cfg, st.stations(cfg))
    assert sig.shape == (cfg.n_pairs,) == (1830,) and sig.min() >= 0.5
