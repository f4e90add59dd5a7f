/* placeholder, replaced by the learned-proposal oracle */
int orc_learned_placeholder(void) { return 0; }
