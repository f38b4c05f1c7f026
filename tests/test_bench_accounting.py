"""The work counts behind bench.py's roofline (host logic, CPU only).

A transform of 2^l points has l layers of n_p/2 butterflies, one GF(2^m)
product each (Alg. 2); a product runs two forward transforms, n_p pointwise
products and one inverse (Alg. 5).  The stages split those layers at the
bottom depth bt: the fused kernel does the low bt layers of all three
transforms plus the pointwise products, the top passes the rest.
"""
import bench


def _products(stage, na, nb, n, field, bt):
    work, kind = bench.stage_work(stage, na, nb, n, 1, field, bt)
    assert kind == "mul"
    return work


def test_products_split_by_depth_add_up_to_alg5():
    for field, na, bt in [(64, 1 << 24, 9), (64, 1 << 30, 11), (128, 1 << 24, 9), (128, 1 << 30, 10)]:
        n = 2 * na
        l = n.bit_length() - 1 - (7 if field == 128 else 6)
        n_p = 1 << l
        total = sum(_products(s, na, na, n, field, bt) for s in ("butterfly", "bottom_fused", "ibutterfly"))
        assert total == 3 * l * (n_p // 2) + n_p                     # three transforms + pointwise
        assert _products("bottom_fused", na, na, n, field, bt) == (3 * bt * (n_p // 2)) + n_p


def test_byte_stages_and_whole_job_value():
    n = 1 << 25
    work, kind = bench.stage_work("encode", 1 << 24, 1 << 24, n, 1)
    assert kind == "hbm" and work == 2 * 2 * n // 8                  # two operands: read n bits, write n_p words
    assert bench.whole_job_value(1000, 2.0, 4, scale=1.0) == 2000.0   # 4 ranks x 1000 units / 2 s


def test_whole_product_alu_counts_alg5_products():
    for field, na in [(64, 1 << 24), (64, 1 << 30), (128, 1 << 30)]:
        n = 2 * na
        l = n.bit_length() - 1 - (7 if field == 128 else 6)
        r = bench.whole_product_alu(n, field, 1.0, 100.0)
        assert r["products"] == 1.5 * l * (1 << l) + (1 << l)
        assert abs(r["frac"] - r["achieved"] / 100.0) < 1e-12


def test_traffic_entry_goes_null_when_the_kernel_changes():
    key = ("bottom_fused", 1 << 30, 1 << 30, 64, 11)
    saved = bench.TRAFFIC_BYTES_PER_LAUNCH[key]
    try:
        bench.TRAFFIC_BYTES_PER_LAUNCH[key] = (123, bench.source_digest(64))
        assert bench.traffic_entry(key, 64)[0] == 123
        bench.TRAFFIC_BYTES_PER_LAUNCH[key] = (123, "0" * 16)
        nbytes, note = bench.traffic_entry(key, 64)
        assert nbytes is None and note.startswith("stale")
    finally:
        bench.TRAFFIC_BYTES_PER_LAUNCH[key] = saved
    assert bench.traffic_entry(("bottom_fused", 5, 5, 64, 1), 64)[0] is None
