"""Which 4- and 5-target tensor-core blocks the planner gives lane-exchange
gathers: an independent statement of the rule the GPU and host tests check
the planner's records against."""


def lane_exchange_expected(n, qubits, ctrls):
    """(layout admits the lane exchange, the automatic rule picks it) for a
    block with these targets and controls (4..6 of them): bit 0 must not be
    a control and the groups must fill tiles of 128; the automatic rule picks
    it for every 5-target block, for 4-target blocks with two or more
    targets among bits 1..3 and for 6-target blocks with one or more."""
    fits = 0 not in ctrls and n - len(qubits) - len(ctrls) >= 7
    low = len(set(qubits) & {1, 2, 3})
    pays = {4: low >= 2, 5: True, 6: low >= 1}[len(qubits)]
    return fits, pays
