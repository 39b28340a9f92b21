"""Host logic of the porosity sweep's model fits (no GPU): rows made to follow
the paper's B_est (Section 4.3) with a known delta_p, and a split layout with
known per-node costs, are fitted back."""
import numpy as np

from paper_2312_14742_gb300.porosity_sweep import fit


def synthetic_rows(delta_p, bmax, s_tile, s_list, n=512 ** 3, cols=22528):
    rows = []
    for phi, full_share, thr_tiled in ((0.2, 0.0, 0.3), (0.5, 0.01, 0.6), (0.8, 0.12, 0.9), (0.95, 0.6, 1.0)):
        nf = int(phi * n)
        empty = int(0.05 * cols * (1 - phi))
        nonempty = cols - empty
        tiled_nodes = int(n * nonempty / cols)
        full_cols = int(full_share * nonempty)
        phi_chunk = nf / tiled_nodes
        r_mixed = (nonempty - full_cols) / nonempty
        b = phi_chunk * bmax / (1 + delta_p * r_mixed / 2)
        t_tiles = 33 * nf / (b * 1e9)
        listed = int(nf * (1 - thr_tiled))
        tiled_split = int(tiled_nodes * thr_tiled)
        info = {"columns": cols, "empty_columns": empty, "full_columns": full_cols, "tiled_nodes": tiled_nodes,
                "listed_nodes": 0, "threshold": 0.0}
        rows.append({
            "porosity": phi, "n_fluid": nf, "n_nodes": n,
            "compact_tiles": {"ms_per_step": t_tiles * 1e3, "compact": info},
            "compact_list": {"ms_per_step": nf * s_list * 1e3, "compact": {"listed_nodes": nf}},
            "compact": {"ms_per_step": (tiled_split * s_tile + listed * s_list) * 1e3,
                        "compact": {"tiled_nodes": tiled_split, "listed_nodes": listed, "threshold": 0.3}},
        })
    return rows


def test_fit_recovers_delta_p_and_rates():
    bmax, s_tile, s_list = 3400.0, 9e-12, 25e-12
    n = 512 ** 3
    full = {"ms_per_step": s_tile * n * 1e3, "bytes_per_node": 33, "B_max_GBps": bmax}
    for delta_p in (0.0, 0.4, 2.5):
        m = fit(synthetic_rows(delta_p, bmax, s_tile, s_list), full)
        assert abs(m["delta_p"] - delta_p) <= 1e-9 + 1e-6 * delta_p
        for b in m["b_est"]:
            assert abs(b["B_est_GBps"] - b["B_fluid_GBps"]) <= 1e-6 * b["B_fluid_GBps"]
        assert abs(m["list_ns_per_node"] - s_list * 1e9) <= 1e-9
        assert abs(m["break_even_fraction"] - s_tile / s_list) <= 1e-9
        for p in m["split_prediction"]:
            assert abs(p["predicted_ms"] - p["measured_ms"]) <= 1e-9 * p["measured_ms"]
